/*
 * carbox.h - C ABI of the GB300 batched astrochemistry solver.
 *
 * The library integrates many independent zero-dimensional gas cells through
 * one mass-action chemical reaction network. The method is the one of the
 * paper "Carbox: an end-to-end differentiable astrochemical simulation
 * framework" (arXiv 2511.10558):
 *
 *   - the network: species and reactions in a uniform format, from which the
 *     incidence (stoichiometry) matrix is built (Sec. 4);
 *   - the ODE  dn_i/dt = +-sum_j k_j n_s1 +- sum_j k_j n_s1 n_s2 (Sec. 2), with
 *     rate coefficients k(phi) of the environment phi = (T, zeta, F_UV, ...)
 *     (Sec. 2: n' = f(n, k(phi), phi));
 *   - rate forms: two-body Kooij-Arrhenius k = alpha (T/300)^beta exp(-gamma/T)
 *     and direct cosmic-ray ionisation k = alpha zeta (Sec. 2); photo-reactions
 *     k = alpha F_UV exp(-gamma A_V) (App. B.1);
 *   - a stiff implicit integrator: variable-order BDF (Sec. 1) with a Newton
 *     iteration on (I - h gamma J) dx = r, J the analytic sparse Jacobian
 *     (Sec. 4 names the sparse/dense trade-off).
 *
 * State and units. The solver integrates x_i = n_i / n_H (abundance per
 * hydrogen nucleus) with n_H constant per cell; two-body coefficients are
 * multiplied by n_H internally. Time is in seconds.
 *
 * Conventions for every function:
 *   - return 0 (CBX_OK) on success, a negative CBX_E* code on error; the
 *     message of the last error on the calling thread is cbx_last_error();
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc,
 *     torch.cuda tensors' data_ptr()); "host pointer" means ordinary memory;
 *   - the caller owns every array it passes; the library owns networks and
 *     its internal workspace;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Device-pointer calls are asynchronous on that stream; errors
 *     found by the host are returned at once, errors of the kernel itself
 *     surface through later CUDA calls as usual.
 *   - arrays of per-cell species values are laid out [S][C], cell index
 *     fastest (x[i*C + c]), species in the order given to cbx_network_create.
 */
#ifndef CARBOX_H
#define CARBOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CBX_VERSION 1

/* error codes (return values) */
#define CBX_OK 0
#define CBX_E_ARG (-1)      /* invalid argument */
#define CBX_E_CUDA (-2)     /* a CUDA call failed; message has the CUDA error */
#define CBX_E_NOMEM (-3)    /* host or device allocation failed */
#define CBX_E_TOO_LARGE (-4) /* network too large for the selected solver */

/* per-cell status codes (cell_status output) */
#define CBX_CELL_OK 0           /* reached t_end */
#define CBX_CELL_MAX_STEPS 1    /* max_steps step attempts used */
#define CBX_CELL_H_UNDERFLOW 2  /* step size fell below 10 ulp(t) */
#define CBX_CELL_BAD_INPUT 5    /* non-finite or non-physical cell parameters */
#define CBX_CELL_TAPE_FULL 6    /* solved, but the trajectory did not fit the tape (no gradient) */

/* reaction types (Sec. 2 and App. B.1) */
#define CBX_TWO_BODY 0    /* A + B -> products, k = alpha (T/300)^beta exp(-gamma/T) */
#define CBX_COSMIC_RAY 1  /* X -> products,     k = alpha zeta                       */
#define CBX_PHOTO 2       /* X -> products,     k = alpha G0 exp(-gamma A_V)         */
#define CBX_CR_PHOTO 3    /* X -> products by secondary photons induced by cosmic
                             rays (App. B.1), k = alpha (T/300)^beta gamma/(1 - omega) zeta:
                             gamma holds the reaction's cosmic-ray efficiency E and
                             omega is the network's grain albedo (cbx_network_set_albedo) */

/* integration method (cbx_options.method) */
#define CBX_METHOD_BDF 0     /* variable-order (1..5) BDF, the field's stiff integrator (Sec. 1) */
#define CBX_METHOD_ESDIRK 1  /* ESDIRK 4(3) of Kvaerno's family, the paper's own kind of solver
                                (Sec. 4); see cbx_esdirk_tableau */

/* precision of the Newton linear algebra */
#define CBX_FP64 0   /* LU, triangular solves and everything else in FP64 */
#define CBX_MIXED 1  /* LU and triangular solves in FP32, FP64 residual r - M dx
                        against the FP64 matrix and iterative refinement; rates,
                        right-hand side, error control and the update stay FP64 */

typedef struct {
  int composition[5]; /* atoms of H, He, C, N, O (used for conservation checks only) */
  int charge;         /* -1, 0, +1 ... */
} cbx_species;

typedef struct {
  int type;     /* CBX_TWO_BODY, CBX_COSMIC_RAY, CBX_PHOTO or CBX_CR_PHOTO */
  int reac[2];  /* reactant species indices; reac[1] = -1 for one-reactant types;
                   reac[0] == reac[1] is A + A (rate kappa x_A^2, A consumed twice) */
  int prod[4];  /* product species indices, -1 = absent; at least one product */
  double alpha, beta, gamma; /* rate parameters of the type's formula */
} cbx_reaction;

typedef struct {
  double n_H;   /* hydrogen nucleus density, cm^-3 (> 0) */
  double T;     /* gas temperature, K (> 0) */
  double A_V;   /* visual extinction, mag */
  double G0;    /* UV field F_UV, Habing units */
  double zeta;  /* cosmic-ray ionisation rate per H2, s^-1 */
} cbx_cell_params;

typedef struct {
  double rtol;        /* relative tolerance (> 0) */
  double atol;        /* absolute tolerance on x (>= 0; rtol*|x| + atol > 0 required) */
  int max_steps;      /* step attempts per cell before CBX_CELL_MAX_STEPS (> 0) */
  int precision;      /* CBX_FP64 or CBX_MIXED */
  int max_refine;     /* CBX_MIXED: refinement sweeps per solve (>= 1) */
  int method;         /* CBX_METHOD_BDF (default) or CBX_METHOD_ESDIRK */
  double refine_tol;  /* CBX_MIXED: stop refining when the weighted RMS of the
                         correction is <= refine_tol */
} cbx_options;

typedef struct {
  int steps;          /* accepted steps */
  int attempts;       /* step attempts (accepted + rejected) */
  int error_fails;    /* rejected by the local error test */
  int newton_fails;   /* rejected because Newton did not converge */
  int rhs_evals;      /* right-hand side evaluations */
  int jac_evals;      /* Jacobian evaluations */
  int lu_factors;     /* LU factorisations of I - cJ */
  int newton_iters;   /* Newton iterations */
  int refine_sweeps;  /* refinement sweeps (CBX_MIXED) */
  int reserved;
  long long t_begin_ns; /* device global timer when the cell's CTA started it */
  long long t_end_ns;   /* device global timer when the cell retired */
} cbx_cell_stats;

typedef struct {
  int S, R;           /* species, reactions */
  int nnz_jac;        /* structural non-zeros of J + I */
  int nnz_lu;         /* non-zeros of the symbolic L + U fill (after ordering) */
  double lu_flops;    /* flops of one numeric LU on that fill */
  double lu_flops_dense; /* 2 S^3 / 3 */
  int smem_bytes_fp64;   /* shared memory per CTA of the FP64 solver (with the sparse
                            pivots' index lists staged when they fit) */
  int smem_bytes_mixed;  /* shared memory per CTA of the mixed solver */
} cbx_netinfo;

typedef struct cbx_network cbx_network;
typedef struct cbx_tape cbx_tape;
typedef struct cbx_server cbx_server;

/* Version of this ABI (CBX_VERSION). */
int cbx_version(void);

/* Message of the last error on the calling thread ("" if none). */
const char* cbx_last_error(void);

/*
 * Build a network: the incidence matrix (Sec. 4), the analytic Jacobian's
 * sparsity pattern, a fill-reducing ordering (minimum degree on the pattern of
 * J + J^T), the symbolic LU fill of I - cJ in that order, and the gather tables
 * of the right-hand side and the Jacobian; then upload them to the current
 * device. Host work, once per network.
 *   species [S], reactions [R]: host pointers, read only during the call.
 *   out: receives a library-owned handle (free with cbx_network_destroy).
 * Errors: CBX_E_ARG for S < 1, R < 0, a bad type, an index out of range, a
 * one-reactant type with two reactants (or the reverse), or no product;
 * CBX_E_CUDA / CBX_E_NOMEM for upload failures.
 */
int cbx_network_create(const cbx_species* species, int S, const cbx_reaction* reactions, int R,
                       cbx_network** out);

/* Free a network (NULL is allowed). The caller makes sure no solve using it is in flight. */
int cbx_network_destroy(cbx_network* net);

/* Sizes and symbolic-analysis figures of a network. */
int cbx_network_info(const cbx_network* net, cbx_netinfo* out);

/*
 * The host compiler's symbolic analysis of a network (Sec. 4 names the sparse
 * structure of the problem), for checks; host memory only, no device access.
 *   perm   [S]    internal -> user species index: the fill-reducing order
 *                 (minimum degree on the pattern of J + J^T); or NULL.
 *   fill   [S*S]  fill[i*S + j] = 1 when entry (i, j), in internal order, of
 *                 the symbolic L + U of I - cJ (static diagonal pivots) is
 *                 structurally non-zero, else 0; or NULL.
 *   kdense        pivots k >= *kdense are factored over full index ranges
 *                 (the dense tail of the FP64 shared-memory LU); or NULL.
 * Errors: CBX_E_ARG for a NULL network.
 */
int cbx_network_symbolic(const cbx_network* net, int* perm, unsigned char* fill, int* kdense);

/* Default options: rtol 1e-4, atol 1e-20, max_steps 100000, CBX_FP64,
   max_refine 5, refine_tol 1e-10, CBX_METHOD_BDF. */
int cbx_default_options(cbx_options* out);

/*
 * The Butcher tableau of CBX_METHOD_ESDIRK, for checks (host memory):
 * a [25] row-major 5 x 5 (lower triangular, a_11 = 0 and a_ii = gamma for
 * i >= 2), c [5], gamma; any pointer may be NULL. The paper's solver is
 * Kvaerno's fifth-order ESDIRK (Sec. 4), whose coefficients it does not print;
 * this is the order-4 member of the same family (Kvaerno, BIT 44, 2004):
 * explicit first stage, stage order 2, embedded order-3 and order-4
 * solutions as stages 4 and 5 (both at c = 1), L-stable; the library derives
 * the coefficients from those conditions (gamma = 0.5728160625).
 * One step: Y_i = y_n + h sum_{j<i} a_ij f(Y_j) + h gamma f(Y_i) (i = 2..5,
 * each by simplified Newton with I - h gamma J), y_{n+1} = Y_5, error
 * estimate Y_5 - Y_4 in the weighted RMS norm, step factor
 * min(10, max(0.2, 0.9 err^(-1/4))).
 */
int cbx_esdirk_tableau(double* a, double* c, double* gamma);

/*
 * Integrate C cells from t0 to t_end (seconds) with the variable-order BDF
 * (or the ESDIRK of cbx_esdirk_tableau when opt->method is CBX_METHOD_ESDIRK;
 * that method has no adjoint: recording entry points reject it).
 *   phi    [C]     device pointer, cell parameters (Sec. 2: k(phi)).
 *   x0     [S][C]  device pointer, initial abundances per n_H.
 *   opt            host pointer (NULL = defaults).
 *   x_out  [S][C]  device pointer, x(t_end) per n_H (may alias nothing else).
 *   cell_status [C] device pointer, CBX_CELL_* per cell.
 *   stats  [C]     device pointer or NULL, per-cell counters.
 * A failing cell never stops the others: it ends with its status and its last
 * accepted state in x_out. Results of a cell do not depend on C, on the other
 * cells, or on the launch configuration (bitwise).
 * Errors: CBX_E_ARG (C < 0, NULL arrays with C > 0, t_end < t0, bad options),
 * CBX_E_TOO_LARGE (the cell's matrix does not fit the solver), CBX_E_CUDA.
 */
int cbx_solve(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
              double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
              cbx_cell_stats* stats);

/*
 * cbx_solve with a time-dependent environment phi(t) per cell (Sec. 2 writes
 * the system as dn/dt = f(n, k(phi), phi); here phi follows a track): the
 * rate coefficients are re-evaluated at every time at which the method
 * evaluates f or J (the step's t_new, and t0 and t0 + h0 at the start).
 *   track [C][K][6]  device pointer, per cell K knots (t_k, n_H, T, A_V, G0,
 *                    zeta), t_k in seconds and strictly increasing; phi(t) is
 *                    linear between knots and takes the end values outside
 *                    [t_0, t_{K-1}]. x is per n_H, so a changing n_H enters
 *                    only the two-body coefficients.
 *   K >= 1           (K = 1: a constant phi, the same result as cbx_solve).
 * Other arguments, ownership and results as for cbx_solve. A cell with a
 * non-finite knot, n_H or T <= 0 at a knot, or knot times not increasing ends
 * with CBX_CELL_BAD_INPUT without touching the others.
 * Errors: those of cbx_solve, and CBX_E_ARG for K < 1 or a NULL track.
 */
int cbx_solve_track(cbx_network* net, const double* track, int K, const double* x0, int C, double t0,
                    double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                    cbx_cell_stats* stats);

/*
 * As cbx_solve, with HOST pointers for phi, x0, x_out, cell_status and stats:
 * the call copies the inputs to the device, solves, copies the results back
 * and synchronises `stream` before returning.
 */
int cbx_solve_host(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                   double t_end, const cbx_options* opt, void* stream, double* x_out,
                   int* cell_status, cbx_cell_stats* stats);

/*
 * Replace the alpha parameters of all reactions (host pointer, R values) in the
 * network, on the host and on its device, for every later solve. Synchronous.
 * Every user of the network sees the change; to solve with other alpha values
 * for one call only (differentiation in ln alpha, Sec. 3), use
 * cbx_solve_with_alpha, which leaves the network unchanged.
 */
int cbx_network_set_alpha(cbx_network* net, const double* alpha);

/*
 * Set the dust grain albedo omega (0 <= omega < 1) of the cosmic-ray-induced
 * photo form (App. B.1: k = alpha (T/300)^beta E/(1 - omega) zeta) for every
 * CBX_CR_PHOTO reaction of the network. A new network has omega = 0. Applies
 * to solves issued after the call. Errors: CBX_E_ARG for a NULL network or
 * omega outside [0, 1).
 */
int cbx_network_set_albedo(cbx_network* net, double omega);

/*
 * Trajectory tape for the adjoint (Sec. 3: gradients of model outputs with
 * respect to chemical and physical inputs; the paper obtains them by automatic
 * differentiation of its solver, here a hand-written discrete adjoint of the
 * BDF map is used).
 * A tape holds, for up to C cells, the program of difference-array operations
 * of the forward solve (initial step, every step-size/order rescale, every
 * accepted step with its result y), plus copies of the cell parameters and
 * initial abundances: the whole forward trajectory is checkpointed, one state
 * per accepted step, so the reverse sweep needs no recomputation.
 *   max_steps: accepted steps a cell may record (cells beyond it end with
 *   CBX_CELL_TAPE_FULL). Device memory: C * (max_steps * (8 S + 8 + 4 * 12) + ...).
 * Library-owned; free with cbx_tape_destroy.
 */
int cbx_tape_create(cbx_network* net, int C, int max_steps, cbx_tape** out);
int cbx_tape_destroy(cbx_tape* tape);

/*
 * cbx_solve that also records the trajectory into `tape` (same arguments as
 * cbx_solve; C must not exceed the tape's capacity). The tape remembers phi,
 * x0, alpha, t0 and t_end for cbx_grad.
 */
int cbx_solve_record(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                     double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                     cbx_cell_stats* stats, cbx_tape* tape);

/*
 * cbx_solve_track that also records the trajectory into `tape` (arguments as
 * cbx_solve_track; C must not exceed the tape's capacity). The tape keeps a
 * copy of the tracks and the time of every accepted step, so that cbx_grad
 * re-evaluates the rate coefficients of phi(t) at each step as the forward
 * solve did. Gradients through a track (cbx_grad / cbx_grad_env):
 *   g_logalpha, g_lnzeta, g_lnG0: as for a constant environment;
 *   g_lognH: derivative with respect to ln of a common factor on the n_H of
 *            every knot of the cell's track;
 *   g_T:     derivative with respect to a common shift (K) of the T of every
 *            knot; g_AV likewise for a common shift of A_V (mag).
 * Errors: those of cbx_solve_track and cbx_solve_record.
 */
int cbx_solve_track_record(cbx_network* net, const double* track, int K, const double* x0, int C, double t0,
                           double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                           cbx_cell_stats* stats, cbx_tape* tape);

/*
 * The time t_new (seconds) of every accepted step recorded for one cell, to
 * the host (for checks); at most cap values. Returns the number of recorded
 * steps (>= 0) or a negative error code. Synchronises the device.
 */
int cbx_tape_step_times(const cbx_tape* tape, int cell, double* t_new, int cap);

/*
 * cbx_solve (tape == NULL) or cbx_solve_record (tape given) with the network's
 * alpha parameters replaced, for this call only, by alpha [R] (device pointer,
 * reaction order of cbx_network_create). The network itself is not changed,
 * so other users of it (other streams, a server, later calls) are not
 * affected: this is how a differentiable solve in ln alpha (Sec. 3:
 * sensitivity to rate coefficients) runs without touching shared state. A
 * tape records the alpha it was solved with; cbx_grad uses that one.
 * Errors: those of cbx_solve / cbx_solve_record, CBX_E_ARG for a NULL alpha.
 */
int cbx_solve_with_alpha(cbx_network* net, const double* alpha, const cbx_cell_params* phi, const double* x0, int C,
                         double t0, double t_end, const cbx_options* opt, void* stream, double* x_out,
                         int* cell_status, cbx_cell_stats* stats, cbx_tape* tape);

/*
 * Discrete adjoint (FP64) of the recorded solve: for the cotangent
 * cot_x = dL/dx(t_end) (device [S][C]) it returns, on `stream`,
 *   g_logalpha [R]  dL/d ln alpha_j summed over cells (device; deterministic order),
 *   g_lognH   [C]  dL/d ln n_H per cell (device),
 *   g_T       [C]  dL/dT per cell, T in K (device).
 * Step sizes and orders are those of the recorded forward solve, and so are
 * the alpha values (the network's at record time, or those passed to
 * cbx_solve_with_alpha); each corrector is differentiated as if solved
 * exactly. Cells whose status was
 * not CBX_CELL_OK get zero gradients. Any output pointer may be NULL.
 */
int cbx_grad(cbx_tape* tape, const double* cot_x, void* stream, double* g_logalpha, double* g_lognH,
             double* g_T);

/*
 * cbx_grad plus the gradients with respect to each cell's radiation and
 * cosmic-ray environment (Sec. 3 asks for sensitivities to physical inputs):
 *   g_lnzeta [C]  dL/d ln zeta: cosmic-ray coefficients are alpha_j zeta (Sec. 2),
 *   g_lnG0   [C]  dL/d ln G0:   photo coefficients are alpha_j G0 exp(-gamma_j A_V)
 *                               (App. B.1),
 *   g_AV     [C]  dL/dA_V (mag), from the same photo form.
 * Each is a fixed-order sum over the cell's per-reaction gradients
 * dL/d ln k_j of the discrete adjoint (device pointers, any may be NULL).
 * Other arguments, ownership and errors as for cbx_grad.
 */
int cbx_grad_env(cbx_tape* tape, const double* cot_x, void* stream, double* g_logalpha, double* g_lognH,
                 double* g_T, double* g_lnzeta, double* g_lnG0, double* g_AV);

/*
 * Read the recorded program of one cell to the host (for checks): kinds
 * (0 init, 1 rescale, 2 step), orders q and values (h0, rho or h); at most cap
 * entries. Returns the number of ops (>= 0) or a negative error code.
 * Synchronises the device.
 */
int cbx_tape_program(const cbx_tape* tape, int cell, int* kinds, int* qs, double* values, int cap);

/*
 * Continuous-batching request server (serving many 0-D cell solves of the
 * Sec. 2 ODE for different networks). A scheduler thread admits submitted
 * requests in arrival order whenever one of `n_streams` CUDA streams and
 * enough of the device-memory budget (inputs, outputs and solver workspace)
 * are free; a request that does not fit may be passed by later, smaller ones
 * at most 8 times, after which nothing else is admitted before it. Queued
 * requests for the same network with the same options and t0 are merged into
 * one launch (up to 65,536 cells), each keeping its own t_end, so that the
 * launch's persistent CTAs back-fill across requests. Admitted launches run
 * concurrently, each with at most `max_ctas` CTAs (0 = the whole device); a
 * cell's solver state stays on chip for its whole solve. Results are bitwise
 * the same whatever else is in flight or merged.
 *   mem_budget: 0 = 80 % of the device memory free at creation; otherwise a
 *               cap, itself limited to that figure.
 * Host arrays are copied at submit (phi [C], x0 [S][C]); cbx_server_wait
 * blocks until the request is done and copies x_out [S][C] and cell_status [C]
 * out (either may be NULL); times (3 doubles, may be NULL) receive the submit,
 * start and completion times in seconds of a steady clock. A request's id is
 * released by cbx_server_wait. cbx_server_poll gives its state (0 queued,
 * 1 running, 2 done, 3 failed) and, when finished, its latency in seconds.
 * cbx_server_info gives the budget in use, the number of launches and how
 * many requests were merged into another's launch.
 * cbx_server_destroy fails the queued requests (their cbx_server_wait returns
 * CBX_E_ARG), waits for the running ones and for every thread blocked in
 * cbx_server_wait, then frees the server; no call may use it afterwards.
 * Errors: CBX_E_ARG, CBX_E_TOO_LARGE (request above the budget or above
 * 65,536 cells), CBX_E_CUDA.
 */
int cbx_server_create(size_t mem_budget, int n_streams, int max_ctas, cbx_server** out);
int cbx_server_submit(cbx_server* server, cbx_network* net, const cbx_cell_params* phi, const double* x0, int C,
                      double t0, double t_end, const cbx_options* opt, uint64_t* request_id);
int cbx_server_poll(cbx_server* server, uint64_t request_id, int* state, double* latency_s);
int cbx_server_wait(cbx_server* server, uint64_t request_id, double* x_out, int* cell_status, double* times);
int cbx_server_stats(cbx_server* server, size_t* peak_bytes, int* peak_running, int* queued);
int cbx_server_info(cbx_server* server, size_t* budget, long long* launches, long long* merged_requests);
int cbx_server_destroy(cbx_server* server);

/*
 * cbx_solve for callers that cannot allocate GPU memory while they run. The
 * paper has no counterpart: this is a deployment variant of cbx_solve with the
 * same arguments, the same kernel and bitwise the same results.
 *
 * cbx_solve takes its scratch (per-CTA rate/Jacobian workspace and a next-cell
 * counter) from the stream-ordered allocator on every call. Hosts that reserve
 * all device memory up front and forbid later allocation by library code,
 * latency-critical loops that must not enter the driver's allocator, and
 * processes running at their memory budget cannot allow that. This entry
 * point calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * is a fixed 16 MiB array compiled into the library, which every GPU that
 * loads the library holds until the process exits.
 *
 * - Set-up: the first call made in a CUDA context (with its device current)
 *   looks up the array's device address (cudaGetSymbolAddress) and caches it
 *   with the context's id; a new context (after cudaDeviceReset, say) gets a
 *   new lookup. Make the first call of each context before any stream capture.
 * - The network's tables must already be on the current device (they are
 *   uploaded by cbx_network_create when a GPU is present); otherwise CBX_E_ARG.
 * - Limit: each CTA needs 8 * (3 R + nnz(J)) bytes of scratch (rounded up to
 *   256 B), plus, for networks whose Newton matrix does not fit in shared
 *   memory (S > 256, e.g. 500 species), the matrix itself:
 *   S * (S | 1) * 8 bytes (CBX_FP64) or * 4 bytes (CBX_MIXED). The number of
 *   CTAs launched is min(C, CTAs the device can run, CTAs that fit in the
 *   16 MiB); for the 500-species / 6000-reaction network that is 7 CTAs
 *   (FP64) or 12 (CBX_MIXED) instead of one per SM, about 20x slower than
 *   cbx_solve, with the same results. Networks the solver cannot run at all
 *   are rejected with CBX_E_TOO_LARGE (within the solver's own limits, S <= 512
 *   and R bounded by shared memory, a CTA needs at most about 5 MB, so every
 *   network that the solver can run fits at least 3 CTAs).
 * - All calls share the one array and it keeps the last call's contents; the
 *   counter is cleared on `stream` at every call (cudaMemsetAsync). Calls
 *   whose kernels overlap on the GPU (other streams, other host threads) race
 *   on the array: issue them on one stream, one after another.
 */
int cbx_solve_noalloc(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                      double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                      cbx_cell_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* CARBOX_H */
