/*
 * stoich.h - C ABI of the GB300 (sm_103a) stoichiometry-matrix chemistry library.
 *
 * The library evaluates, for many independent hydro cells at once, the chemical
 * right-hand side dx/dt = S R(x) of the paper's matrix formulation (Eq. 7, with
 * S the species x reaction stoichiometry matrix and R_j = k'_j prod x_reactants,
 * Eqs. 2-6), its Jacobian J = S dR/dx, and a BDF/Newton stiff integrator that
 * consumes them (the role DLSODES plays in Section 3).
 *
 * Conventions shared by every call:
 *  - Every function returns an sm_status (SM_OK == 0) and never aborts, traps
 *    or exits; sm_status_str() gives a message.
 *  - Batched arrays are species-major (or reaction-major) with the CELL index
 *    fastest: element (i, c) of an [n][ld] array lives at i*ld + c, with
 *    C <= ld.  ld must be a multiple of 32 (coalesced 256-byte rows).
 *  - Pointers named d_* are DEVICE pointers on the network's device, owned by
 *    the caller; the library never frees them.  Pointers named h_* are host
 *    pointers.  Handles (sm_net, sm_state) and their internal device buffers
 *    are owned by the library and released by the matching *_free call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device calls are asynchronous on that stream; errors raised inside a
 *    kernel are written to a device status word and reported by sm_sync() or
 *    by the next synchronous call on the same handle.
 *  - Sizes: C >= 0; C == 0 is a valid no-op.
 */
#ifndef STOICH_H
#define STOICH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sm_status;
enum {
    SM_OK = 0,
    SM_EINVAL = 1,     /* bad argument (null pointer, size, layout, enum)       */
    SM_ENOMEM = 2,     /* device or host allocation failed                      */
    SM_ECUDA = 3,      /* a CUDA runtime call failed                            */
    SM_ENOTCONS = 4,   /* network does not conserve elements / charge (E.S!=0)  */
    SM_ETIMEOUT = 5,   /* a bounded device wait ran out                         */
    SM_EPARTIAL = 6,   /* the call completed but some cells failed (see stats)  */
    SM_ENOTSUP = 7,    /* combination not supported                             */
    SM_ETOOBIG = 8     /* request exceeds a fixed-size internal buffer          */
};

/* Per-cell integration status (sm_cell_stats.status). */
enum {
    SM_CELL_OK = 0,
    SM_CELL_MAXSTEPS = 1,  /* max_steps accepted steps taken before t_end       */
    SM_CELL_HMIN = 2,      /* step size fell below the time resolution          */
    SM_CELL_CONV = 3,      /* repeated Newton convergence failures              */
    SM_CELL_NAN = 4,       /* non-finite input or state                         */
    SM_CELL_RUNNING = 5    /* not finished yet (integration continues)          */
};

/* Reaction classes and their rate laws (rates are evaluated once per cell,
 * outside the solver, as in Section 3):
 *   SM_TWO_BODY, SM_DISS_RECOMB: k = alpha (T/300)^beta exp(-gamma/T), k' = k n_H
 *   SM_COSMIC_RAY:               k = alpha zeta,                        k' = k
 *   SM_PHOTO:                    k = alpha exp(-gamma A_V),             k' = k   */
enum { SM_TWO_BODY = 0, SM_COSMIC_RAY = 1, SM_PHOTO = 2, SM_DISS_RECOMB = 3 };

/* Storage formats of S (Section 2.2, Listings 1-4) and row orders (Section 3). */
enum { SM_FMT_CRS = 0, SM_FMT_COO = 1, SM_FMT_CCS = 2, SM_FMT_SELL = 3 };
enum { SM_ORDER_NONE = 0, SM_ORDER_NNZ = 1, SM_ORDER_RCM = 2 };

/* Explicit network description (host arrays, read during sm_net_build only).
 *   comp      int32 [n_s][n_elem+1]: atoms of each element, last column = charge
 *   reactants int32 [n_r][2]: species indices, -1 padded (first entry >= 0);
 *             a species listed twice reacts with multiplicity two
 *   products  int32 [n_r][4]: species indices, -1 padded
 *   rclass    int8  [n_r]: SM_TWO_BODY ... SM_DISS_RECOMB
 *   alpha, beta, gamma double [n_r]: rate parameters (see the class enum)   */
typedef struct {
    int32_t n_s, n_r, n_elem;
    const int32_t* comp;
    const int32_t* reactants;
    const int32_t* products;
    const int8_t* rclass;
    const double* alpha;
    const double* beta;
    const double* gamma;
} sm_net_desc;

typedef struct sm_net sm_net;

/* Network statistics and per-cell algorithmic work of the batched kernels. */
typedef struct {
    int32_t n_s, n_r;
    int64_t nnz_S;          /* nonzeros of S (net coefficients)                 */
    int64_t nnz_J;          /* structural nonzeros of J, diagonal included      */
    int64_t n_jac_terms;    /* sum over J entries of contributing reactions     */
    int64_t nnz_LU;         /* nonzeros of L+U after symbolic factorisation     */
    int64_t lu_flops;       /* flops of one numeric factorisation (2 per FMA)   */
    int32_t lu_head;        /* pivots eliminated as sparse before the dense tail */
    int32_t max_row_nnz;    /* longest row of S (the H row in the paper)        */
    int32_t fmt, order, sell_C, sell_sigma; /* current traversal format        */
    int64_t fmt_entries;    /* stored entries of the current format (pads incl.) */
    double rhs_bytes;       /* per cell: 8 (n_r + 2 n_s)                        */
    double rhs_flops;       /* per cell: 2 nnz_S + sum_j order_j                */
    double jac_bytes;       /* per cell: 8 (n_r + n_s + nnz_J)                  */
    double jac_flops;       /* per cell: 2 n_jac_terms + sum_j order_j          */
    int64_t lu_packed;      /* values per cell of the factors as the integrator's
                               substitution reads them (sparse head parts + the
                               dense trailing block, column-major, padded)     */
} sm_net_info;

/* Build a network on `device` from an explicit description: validates indices
 * and classes (SM_EINVAL) and conservation E.S = 0 (SM_ENOTCONS); builds S
 * (Eq. 7: products minus reactants, zero net entries dropped), the traversal
 * formats, the Jacobian pattern and the symbolic LU, and uploads them once.
 * The default traversal is CRS in the original order.  *out receives a handle
 * owned by the caller until sm_net_free. */
sm_status sm_net_build(const sm_net_desc* d, int32_t device, sm_net** out);
sm_status sm_net_free(sm_net* net);

/* Seeded synthetic network of the paper's shape (the UMIST network of Section
 * 3 is not distributed): species from H, C, O and e- (neutral, cationic and
 * small anionic compositions, small first, alphabetical by formula), reactions
 * grouped by class 60 % two-body, 20 % cosmic ray, 15 % photo, 5 % dissociative
 * recombination, each with 1-2 reactants and 1-4 products conserving every
 * element and the charge; two-body / DR log10 alpha ~ U[-12,-9], beta ~
 * U[-1,1], gamma ~ U[0,500] K; cosmic ray log10 alpha ~ U[0,3]; photo log10
 * alpha ~ U[-11,-9], gamma ~ U[1,3].  Every draw comes from counter-based
 * SplitMix64 streams of `seed`, so the arrays are identical on every platform.
 * sm_synth_network fills caller-owned host arrays in the layout of
 * sm_net_desc (comp [n_s][4], reactants [n_r][2], products [n_r][4] padded with
 * -1, rclass, alpha, beta, gamma [n_r]); sm_net_build_synthetic builds the
 * network from them (as sm_net_build with n_elem = 3).  SM_EINVAL if n_s < 12,
 * n_r < 1, an array is NULL, or the species set cannot hold n_r distinct
 * reactions. */
sm_status sm_synth_network(uint64_t seed, int32_t n_s, int32_t n_r, int32_t* comp, int32_t* reactants,
                           int32_t* products, int8_t* rclass, double* alpha, double* beta, double* gamma);
sm_status sm_net_build_synthetic(uint64_t seed, int32_t n_s, int32_t n_r, int32_t device, sm_net** out);

/* Select the traversal used by sm_rhs_eval: fmt (SM_FMT_*), row order
 * (SM_ORDER_*; nnz = descending nonzero count, stable, Section 3; RCM =
 * reverse Cuthill-McKee on pattern(S S^T)), and for SELL the slice height C
 * (1..32) and sorting window sigma (>= 1).  Results do not depend on the
 * choice beyond floating-point summation order. */
sm_status sm_net_set_format(sm_net* net, int32_t fmt, int32_t order, int32_t sell_C,
                            int32_t sell_sigma);
sm_status sm_net_get_info(const sm_net* net, sm_net_info* info);

/* Select the integrator's right-hand-side gather (run in every Newton
 * iteration): CRS in row order `order` (SM_ORDER_*) with 8, 16 or 32 cells per
 * CTA.  sm_net_autotune makes this choice by measurement; the default is the
 * original order with 16 cells.  States keep the choice current when they
 * capture their graph of attempts.  SM_EINVAL on other values. */
sm_status sm_net_set_integ(sm_net* net, int32_t order, int32_t cells_per_cta);

/* Result of sm_net_autotune. */
typedef struct {
    int32_t fmt, order, sell_C, sell_sigma;  /* the selected traversal          */
    double us;                               /* its median sm_rhs_eval time     */
    int32_t candidates;                      /* traversals timed (0 if cached)  */
    int32_t cached;                          /* 1: taken from the process cache */
    int32_t integ_order;                     /* the integrator's gather: row order */
    int32_t integ_cells_per_cta;             /*   and cells per CTA (8, 16, 32)    */
    double integ_us;                         /*   its median time (rate pass + gather) */
} sm_tune_result;

/* Measured choice of the sm_rhs_eval traversal (the paper's storage-format
 * comparison, Section 3, done per network and GPU): builds each candidate of
 * a fixed grid (CRS, COO, CCS x row orders; SELL-C-sigma with C in {4, 8, 32}
 * and sigma in {1, 8C, n_s}), runs sm_rhs_eval on the caller's device arrays
 * d_k = k'[n_r][ld], d_y = x[n_s][ld] (C cells) writing d_f = f[n_s][ld], times
 * one warm-up and five calls with CUDA events on `stream` (median), and leaves
 * the fastest selected (as sm_net_set_format would).  It then times the
 * integrator's Newton-iteration right-hand side (rate pass + masked CRS
 * gather) for CRS in each row order x 8, 16 or 32 cells per CTA on the same
 * inputs and selects the fastest for the network's integrations; a state
 * keeps the choice that was current when it captured its graph of attempts,
 * so tune before integrating.  The choice is cached for
 * the process per (network content, device name, C rounded up to a power of
 * two); force = 1 measures again.  Synchronises with `stream`.  d_f is
 * scratch: it holds the last candidate's result on return.  If a candidate
 * fails (SM_ENOMEM, SM_ECUDA), the traversal selected before the call is
 * restored and the error returned.  SM_EINVAL on bad arguments or a
 * host-only network. */
sm_status sm_net_autotune(sm_net* net, int64_t C, const double* d_k, const double* d_y, double* d_f,
                          int64_t ld, int32_t force, void* stream, sm_tune_result* out);

/* Export host copies of internal structures for bit-exact checks.  what:
 *  SM_X_ROW_ORDER int32[n_s]    rows (species) in traversal order
 *  SM_X_COL_ORDER int32[n_r]    columns (reactions) in traversal order
 *  SM_X_FMT_PTR   int32[]       CRS row_ptr / CCS col_ptr / SELL slice_ptr (COO: none)
 *  SM_X_FMT_IDX   int32[]       CRS col_ind / CCS row_ind / COO row_ind / SELL col_ind
 *  SM_X_FMT_IDX2  int32[]       COO col_ind / SELL row_id (-1 = padding row)
 *  SM_X_FMT_VAL   double[]      coefficients (0 at SELL pads)
 *  SM_X_FMT_LEN   int32[]       SELL slice lengths
 *  SM_X_JPAT_PTR  int32[n_s+1]  CRS row pointer of the Jacobian pattern
 *  SM_X_JPAT_COL  int32[nnz_J]  its column indices (ascending per row)
 *  SM_X_LU_PERM   int32[n_s]    elimination order of the Newton matrix
 * sm_net_export_size() returns the byte size; sm_net_export() copies exactly
 * that many bytes into h_buf (SM_EINVAL if `bytes` is smaller). */
enum {
    SM_X_ROW_ORDER = 0, SM_X_COL_ORDER = 1, SM_X_FMT_PTR = 2, SM_X_FMT_IDX = 3,
    SM_X_FMT_IDX2 = 4, SM_X_FMT_VAL = 5, SM_X_FMT_LEN = 6, SM_X_JPAT_PTR = 7,
    SM_X_JPAT_COL = 8, SM_X_LU_PERM = 9
};
sm_status sm_net_export_size(const sm_net* net, int32_t what, size_t* bytes);
sm_status sm_net_export(const sm_net* net, int32_t what, void* h_buf, size_t bytes);

/* Rate coefficients k'[n_r][ld] (FP64) for C cells with temperature d_T[C] (K),
 * density d_nH[C] (cm^-3) and visual extinction d_Av[C]; zeta is the
 * cosmic-ray ionisation rate (s^-1).  Rate laws: see the class enum.  Computed
 * as exp(log alpha + beta log(T/300) - gamma/T) n_H for two-body classes, so
 * results differ from alpha (T/300)^beta exp(-gamma/T) n_H by rounding only. */
sm_status sm_rates_eval(const sm_net* net, int64_t C, const double* d_T, const double* d_nH,
                        const double* d_Av, double zeta, double* d_k, int64_t ld, void* stream);

/* sm_rates_eval with a per-cell FUV field: d_chi[C] (device; NULL = 1 in every
 * cell) multiplies the photorates, k = chi alpha exp(-gamma A_V), the
 * illumination of the paper's PDR benchmark (chi = 1e5 Draine fields,
 * Section 3).  Other classes as in sm_rates_eval. */
sm_status sm_rates_eval_chi(const sm_net* net, int64_t C, const double* d_T, const double* d_nH,
                            const double* d_Av, const double* d_chi, double zeta, double* d_k, int64_t ld,
                            void* stream);

/* Right-hand side f = S R(y) (Eq. 7) for C cells: d_k = k'[n_r][ld], d_y =
 * x[n_s][ld] -> d_f[n_s][ld], FP64, with the traversal chosen by
 * sm_net_set_format.  d_f must not alias d_k or d_y. */
sm_status sm_rhs_eval(const sm_net* net, int64_t C, const double* d_k, const double* d_y,
                      double* d_f, int64_t ld, void* stream);

/* Right-hand side without any device allocation.  Same inputs, outputs,
 * formats and results as sm_rhs_eval, for callers that cannot let a library
 * call cudaMalloc: hydro codes that reserve the device memory up front for
 * their own pool allocator (an allocation from inside the chemistry call
 * would fail or take memory the pool counts on), and codes whose time-step
 * loop must not allocate because cudaMalloc can synchronise the device.  The
 * per-reaction rate buffer lives in one fixed array compiled into the library
 * (SM_STATIC_SCRATCH_DOUBLES doubles, 32 MiB, held by every GPU that loads
 * the library until the process exits); requests with
 * n_r * round_up(C, 32) > SM_STATIC_SCRATCH_DOUBLES return SM_ETOOBIG.
 * The first call on a device looks up that array's device address (a
 * set-up step done once per device), so make that first call before any
 * stream capture.  Every call on a device shares the array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The array keeps the last call's contents;
 * nothing in it needs to start at zero because each call writes every value
 * it reads.  The paper has no counterpart to this entry point. */
#define SM_STATIC_SCRATCH_DOUBLES 4194304
sm_status sm_rhs_eval_static(const sm_net* net, int64_t C, const double* d_k, const double* d_y,
                             double* d_f, int64_t ld, void* stream);

/* Jacobian values J = S dR/dx on the static pattern (SM_X_JPAT_*): d_J is
 * [nnz_J][ld], entry p of the pattern for cell c at p*ld + c, FP64. */
sm_status sm_jac_eval(const sm_net* net, int64_t C, const double* d_k, const double* d_y,
                      double* d_J, int64_t ld, void* stream);

/* ------------------------------------------------------------------------
 * Stiff integration (the role of DLSODES in Section 3): a variable-step,
 * variable-order (1..5) BDF method with simplified Newton iterations, run
 * independently for every cell.  The method, step-size / order rules and
 * Jacobian-refresh policy are fixed (see the option fields):
 *  - order-q BDF on the last q solution points with Lagrange coefficients,
 *    degree-q Lagrange predictor (y0 + h f(y0) on the first step);
 *  - Newton matrix M = I - gamma J (gamma = h / alpha_0), J evaluated at the
 *    predicted state, refreshed at the first attempt, after j_age_max steps,
 *    when gamma moved by more than gamma_tol relative, and after a Newton
 *    failure that used an older J; corrections scaled by 2/(1+gamma/gamma_J);
 *  - convergence when |delta|_wrms * min(1, rate) <= newton_tol (rate =
 *    max(0.3 rate, |delta_m|/|delta_m-1|)), at most newton_max iterations;
 *  - error estimate h/(t_{n+1}-t_{n-q}) |y - y_pred|_wrms, step factor
 *    0.9 err^(-1/(q+1)) clipped to [0.2, eta_max] (1 after a rejection),
 *    factors in [1, eta_keep) ignored; neighbouring orders rated after q+1
 *    steps at order q.  |v|_wrms = sqrt(mean((v_i/(rtol|y_i|+atol))^2)).
 * The Newton matrix is factorised without pivoting in a minimum-degree order
 * (as DLSODES's sparse solver does); SM_PREC_FP64 factorises and solves in
 * FP64, SM_PREC_MIXED in FP32 on the WRMS-equilibrated matrix W M W^-1
 * while the residual, Jacobian and all state stay FP64; SM_PREC_TF32 is
 * SM_PREC_MIXED with the dense trailing block's updates on the tensor cores
 * (each operand split into TF32 high and low parts, three products per pair,
 * FP32 accumulation: FP32-level accuracy).  In both reduced precisions
 * each Newton iteration forms an FP64 residual, so the iteration refines the
 * low-precision solve.
 * ------------------------------------------------------------------------ */
enum { SM_PREC_FP64 = 0, SM_PREC_MIXED = 1, SM_PREC_TF32 = 2 };

typedef struct {
    double rtol, atol;        /* error weights 1/(rtol |y| + atol)                 */
    double gamma_tol;         /* refactor when |gamma/gamma_J - 1| > gamma_tol     */
    double newton_tol;        /* Newton convergence threshold (WRMS units)         */
    double eta_max;           /* largest step growth factor                        */
    double eta_keep;          /* growth factors in [1, eta_keep) are not applied   */
    int32_t q_max;            /* highest BDF order, 1..5                           */
    int32_t max_steps;        /* accepted steps per cell before SM_CELL_MAXSTEPS   */
    int32_t j_age_max;        /* accepted steps between Jacobian refreshes         */
    int32_t newton_max;       /* Newton iterations per attempt, 1..8               */
    int32_t max_conv_fails;   /* consecutive Newton failures before SM_CELL_CONV   */
    int32_t precision;        /* SM_PREC_FP64, SM_PREC_MIXED or SM_PREC_TF32       */
    int32_t use_graph;        /* capture the attempt loop in a CUDA graph (1) or not */
    int32_t attempts_per_sync;/* attempts launched between completion checks      */
    int32_t timing_kind;      /* SM_TIME_*: kernel class timed with CUDA events    */
    int32_t record_steps;     /* > 0: record up to this many accepted steps per cell
                                 (times, sizes, orders) and the step history every
                                 SM_CHECKPOINT_EVERY steps, for sm_adjoint         */
    int32_t refresh_ctas_per_sm; /* refresh CTAs resident per SM: 0 = as many as
                                 fit (default); fewer CTAs keep fewer working
                                 matrices in flight (L2 footprint)            */
} sm_opts;

/* Accepted steps between stored states of the recorded forward run. */
#define SM_CHECKPOINT_EVERY 16

/* Kernel classes of the integrator whose launches sm_state_timing reports. */
enum { SM_TIME_NONE = 0, SM_TIME_REFRESH = 1, SM_TIME_RHS = 2, SM_TIME_SOLVE = 3,
       SM_TIME_PREDICT = 4, SM_TIME_FINISH = 5 };

/* Per-cell result of sm_integrate (device array of C entries). */
typedef struct {
    int32_t status;        /* SM_CELL_*                                      */
    int32_t steps;         /* accepted steps                                 */
    int32_t rejects;       /* error-test failures                            */
    int32_t conv_fails;    /* Newton convergence failures                    */
    int32_t newton_iters;  /* Newton iterations (RHS evaluations after init) */
    int32_t jac_evals;     /* Jacobian evaluations = factorisations          */
    int32_t q_last;        /* order at the end                               */
    int32_t pad;
    double t;              /* time reached                                   */
    double h;              /* next step size                                 */
} sm_cell_stats;

typedef struct sm_state sm_state;

/* Defaults: rtol 1e-6, atol 1e-20, gamma_tol 0.3, newton_tol 0.1, eta_max 5,
 * eta_keep 1.5, q_max 5, max_steps 100000, j_age_max 20, newton_max 4,
 * max_conv_fails 10, FP64, graph on, 8 attempts per completion check. */
void sm_opts_default(sm_opts* o);

/* Integrator workspace for up to C cells of `net` (library-owned device
 * memory: history, Newton vectors and one factorised Newton matrix per cell,
 * n_s^2 values in the chosen precision).  SM_ENOMEM if it does not fit. */
sm_status sm_state_create(const sm_net* net, int64_t C, const sm_opts* opts, sm_state** out);
sm_status sm_state_free(sm_state* st);
/* Bytes of device memory the state holds. */
sm_status sm_state_bytes(const sm_state* st, size_t* bytes);

/* Integrate C cells (C <= the state's capacity) from t = 0 to t_end (s):
 * d_k = k'[n_r][ld] rate coefficients, d_y = x[n_s][ld] initial abundances,
 * overwritten with the abundances at t_end (or where a cell stopped).
 * d_stats (device, C entries, may be NULL) receives per-cell results.
 * Returns SM_EPARTIAL if any cell did not reach t_end. */
sm_status sm_integrate(sm_state* st, int64_t C, const double* d_k, double* d_y, int64_t ld,
                       double t_end, sm_cell_stats* d_stats, void* stream);

/* Stepwise use: sm_state_init sets t = 0 from d_y; each sm_step_bdf call runs
 * `attempts` BDF attempts (predict, Newton, error test) for every unfinished
 * cell toward t_end; sm_state_read copies the current solution to d_y and the
 * per-cell results to d_stats (either may be NULL) and reports how many cells
 * are still running in *h_running (host, may be NULL; synchronises). */
sm_status sm_state_init(sm_state* st, int64_t C, const double* d_k, const double* d_y, int64_t ld,
                        double t_end, void* stream);
sm_status sm_step_bdf(sm_state* st, const double* d_k, int64_t ld, int32_t attempts, void* stream);
sm_status sm_state_read(sm_state* st, double* d_y, int64_t ld, sm_cell_stats* d_stats,
                        int64_t* h_running, void* stream);

/* Checkpoint / resume of an integration.  sm_state_save writes an image of
 * the state (per-cell time, step size, order, counters and status, the step
 * history and working vectors, the step records, and with with_factors = 1
 * the factorised Newton matrices) into the caller's host buffer; *needed
 * receives the image size (call with host = NULL to query it; the factors are
 * n_s x ldm values per cell of capacity, FP32 or FP64).  sm_state_load puts an
 * image back into a state created for the same network size, capacity,
 * precision and record length (SM_EINVAL otherwise); stepping it then
 * continues the saved integration with the loading state's options.  With the
 * factors the continuation is bit-identical to an uninterrupted run; without
 * them every cell refactorises its Newton matrix on its next attempt.  Both
 * synchronise with the state's stream before returning. */
sm_status sm_state_save(sm_state* st, int32_t with_factors, void* host, size_t bytes, size_t* needed,
                        void* stream);
sm_status sm_state_load(sm_state* st, const void* host, size_t bytes, void* stream);

/* Instrumentation: *launches = kernels the state has launched so far, and,
 * when opts.timing_kind selects a class, *ms = summed CUDA-event durations of
 * that class's launches (*timed = how many were timed; the RHS class times
 * the rate + gather pair of each Newton round as one launch).  Events are
 * recorded on the state's stream, inside the captured graph when graphs are
 * used; sm_state_timing_reset zeroes the totals.  Any pointer may be NULL. */
sm_status sm_state_timing(const sm_state* st, int64_t* launches, double* ms, int64_t* timed);
sm_status sm_state_timing_reset(sm_state* st);

/* ---- Coupled gas temperature ---------------------------------------------
 * The paper holds T fixed inside a chemistry step and updates the energy
 * outside the chemical solver (Section 5).  A network given a temperature
 * slot by sm_net_set_thermal integrates T as one more component of the same
 * implicit BDF system.  Slot t is a species with no atoms, no charge and no
 * reactions whose value is the gas temperature in K; with x_tot the sum of
 * the other components (electrons included) and f = S R(k'(T), x) (Eq. 7),
 *   3/2 x_tot dT/dt = heat - n_H sum_i x_i L_i exp(-E_i / T)
 *                     - lam n_H (T - T_dust) - 3/2 T sum_{i != t} f_i,
 * i.e. the thermal energy 3/2 T x_tot per H nucleus gains a constant heating,
 * loses two-level line cooling and gas-grain exchange, and follows the
 * particle number.  The two-body and dissociative-recombination
 * coefficients k' (the T-dependent classes) are re-evaluated from the state's
 * T before every right-hand side; the cosmic-ray and photo ones once, at
 * sm_state_init.  The Newton matrix keeps the species block's sparse LU and
 * adds T by block elimination: per refresh one more substitution
 * (z = M^-1 (-gamma dF/dT)) and a scalar Schur complement, per Newton
 * iteration one dot product and one update; the result is the solution of
 * the full (n_s) x (n_s) system with T eliminated last.
 *
 * sm_net_set_thermal: th = NULL turns the mode off.  L and E are host arrays
 * of n_s values (copied): L_i >= 0 in K cm^3 s^-1 (0: not a coolant), E_i > 0
 * in K where L_i > 0.  heat (K s^-1 per H nucleus), lam (cm^3 s^-1), T_dust
 * (K) and zeta (s^-1, the cosmic-ray rate of the rate laws) >= 0.  SM_EINVAL
 * if slot t has atoms or charge or appears in a reaction.  States created
 * from the network afterwards take a copy of the setting; a thermal state
 * records steps (sm_state_steps) but has no adjoint or replay and cannot be
 * saved or loaded (SM_ENOTSUP), and needs the cells' conditions from
 * sm_state_set_cells before sm_state_init / sm_integrate; its d_k arguments
 * are ignored and may be NULL. */
typedef struct {
    int32_t t_index;       /* species slot holding T (K)                            */
    double heat;           /* constant heating per H nucleus, K s^-1                */
    double lam;            /* gas-grain coupling coefficient, cm^3 s^-1             */
    double T_dust;         /* dust temperature, K                                   */
    double zeta;           /* cosmic-ray ionisation rate of the rate laws, s^-1     */
    const double* L;       /* host [n_s]: line-cooling coefficients, K cm^3 s^-1    */
    const double* E;       /* host [n_s]: excitation temperatures, K                */
} sm_thermal;
sm_status sm_net_set_thermal(sm_net* net, const sm_thermal* th);

/* Per-cell conditions of a thermal state: n_H (cm^-3), A_V and the FUV
 * field chi (d_chi may be NULL: 1) for cells 0..C-1, device arrays of C
 * doubles, copied on `stream` into the state (C <= capacity).  SM_ENOTSUP on
 * a state without a temperature slot. */
sm_status sm_state_set_cells(sm_state* st, int64_t C, const double* d_nH, const double* d_Av,
                             const double* d_chi, void* stream);

/* ---- Sensitivities: discrete adjoint of the BDF integration -----------------
 * The paper integrates the network but computes no derivatives; these calls
 * are the library's addition.  They differentiate the frozen-step map of the
 * last recorded run (opts.record_steps > 0): the accepted steps (t_m, h_m,
 * q_m), m = 1..N, are held fixed and every implicit BDF equation
 *   alpha_0^m y_m + sum_{i=1..q_m} alpha_i^m y_{m-i} - h_m f(y_m; k) = 0
 * (alpha from the step times, as in the integrator) is taken as solved
 * exactly.  For Phi = c^T y_N, backwards in m,
 *   (alpha_0^m I - h_m J(y_m))^T lambda_m = c [m = N] - sum_{m'} alpha_{m'-m}^{m'} lambda_{m'}
 * over the later steps m' with m' - m <= q_{m'}, and
 *   dPhi / d log k_j = sum_m h_m R_j(y_m) (S^T lambda_m)_j
 * because f = S R (Eq. 7) and each R_j is proportional to k_j. */

/* Largest number of cotangents per sm_adjoint call. */
#define SM_ADJ_MAX_COT 64

/* Copies the recorded step log of the state's last run: d_t[m][ld] = t_m (end
 * time of accepted step m + 1), d_h[m][ld] = h_m, d_q[m][ld] = order, for
 * m < m_max <= opts.record_steps (device arrays; rows past a cell's step
 * count are unspecified; the per-cell count is sm_cell_stats.steps).
 * SM_EINVAL if the state records nothing or m_max is out of range. */
sm_status sm_state_steps(sm_state* st, int32_t m_max, double* d_t, double* d_h, int32_t* d_q, int64_t ld,
                         void* stream);

/* Reverse sweep for n_cot cotangents at once (1 <= n_cot <= SM_ADJ_MAX_COT).
 * d_k     = the k'[n_r][ld] the recorded run was integrated with (device);
 * d_cot   = c[n_cot][n_s][ld] (device), the weights of y_N for each Phi;
 * d_grad  = out[n_cot][n_r][ld] (device): dPhi_v / d log k_j per cell;
 * d_grad_y0 = out[n_cot][n_s][ld] (device, may be NULL): dPhi_v / dy_0, the
 *           recursion continued to the initial state, which enters the first
 *           steps' equations through alpha_{m'}^{m'} y_0 (m' <= q_{m'});
 * d_astat = per-cell status (device, C entries, may be NULL): 0 ok, 1 no
 *           usable record (the cell did not finish with SM_CELL_OK or took
 *           more than opts.record_steps steps; its gradient is 0), 2 a
 *           recomputed step's Newton iteration did not reach its tolerance
 *           (the gradient is computed but less accurate).
 * Work and memory: segments of SM_CHECKPOINT_EVERY steps are recomputed from
 * the stored step history (last first), each recomputed state gets its own
 * FP64 factorisation, then the segment is swept backwards.  The workspace is
 * library-owned, grown on the first call and kept with the state: about
 * SM_CHECKPOINT_EVERY * n_s * ldm * 8 bytes per cell of a pass (ldm = n_s
 * rounded up to a multiple of 8) plus the cotangent vectors; cells_per_pass
 * (0 = all cells in one pass; otherwise rounded up to a multiple of 32)
 * bounds it.  The call overwrites the integrator's working vectors (the
 * history): read the solution first, and call sm_state_init or sm_integrate
 * before stepping again; recorded steps and sm_cell_stats stay valid.
 * Errors: SM_EINVAL (bad arguments, or the state records nothing),
 * SM_ENOTSUP (a state created with SM_PREC_MIXED or SM_PREC_TF32: the adjoint runs in FP64
 * only), SM_ENOMEM (workspace does not fit: use a smaller cells_per_pass);
 * SM_EPARTIAL if any cell's d_astat is not 0.  Synchronises the host with the
 * state's stream once per pass. */
sm_status sm_adjoint(sm_state* st, const double* d_k, int64_t ld, const double* d_cot, int32_t n_cot,
                     double* d_grad, double* d_grad_y0, int32_t* d_astat, int64_t cells_per_pass,
                     void* stream);

/* Frozen-step replay: re-solves the recorded run's accepted steps (same t_m,
 * h_m, q_m) from its recorded initial state with other rate coefficients d_k
 * (k'[n_r][ld], device) and writes y_N to d_y (x[n_s][ld], device; NaN for
 * cells without a usable record).  Each implicit step is solved by Newton to
 * 1e-4 in the run's WRMS norm, with the Newton matrix refreshed when h/alpha_0
 * moves by more than opts.gamma_tol and every SM_CHECKPOINT_EVERY steps.  This
 * is the map sm_adjoint differentiates, so central differences of it check
 * the adjoint.  d_astat, cells_per_pass, the errors and the effect on the
 * state's working vectors are those of sm_adjoint (no factor slots are used:
 * the workspace is the cotangent-free part). */
sm_status sm_replay(sm_state* st, const double* d_k, int64_t ld, double* d_y, int32_t* d_astat,
                    int64_t cells_per_pass, void* stream);

/* Measured arithmetic throughput of the device's FMA pipes (the ceilings
 * of the FP64-bound right-hand side, Jacobian and residual and of the
 * FP32 factorisation, Section 5's roofline analysis carried to this GPU):
 * fp64 = 1 probes FP64, 0 probes FP32.  Every thread of several CTAs per SM
 * runs eight independent FMA chains (2 flops each), timed with CUDA events
 * over three launches after a warm-up; *tflops receives the best rate in
 * TFLOP/s.  Allocates and frees a small device buffer, synchronises the
 * device's legacy stream.  SM_EINVAL on a NULL pointer or negative device. */
sm_status sm_probe_fma(int32_t device, int32_t fp64, double* tflops);

/* Per-phase cycle counters of the Newton-matrix refresh (a diagnostic for
 * profiling; the library must be built with the phase-clock option, see the
 * package's build.py, otherwise SM_ENOTSUP).  h_out receives 16 doubles:
 * slots 0-10 the clock64() cycles summed over all CTAs of `device` for the
 * phases zero / dR / weights, Jacobian gather and M, sparse head, head
 * Schur complement, head packing, panel loads, panel LU, U block load, U
 * block solve, trailing update, epilogue; slot 15 the refreshed cells.
 * reset = 1 zeroes the counters after reading them. */
sm_status sm_phase_cycles(int32_t device, double* h_out, int32_t reset);

/* Wait for all work on `stream` and report (and clear) any error a kernel of
 * this network wrote to its device status word. */
sm_status sm_sync(const sm_net* net, void* stream);

const char* sm_status_str(sm_status s);

#ifdef __cplusplus
}
#endif
#endif /* STOICH_H */
