/*
 * gamesolve.h - C ABI of the GB300 policy-iteration / algebraic-multigrid
 * solver for discounted two-player zero-sum stochastic games.
 *
 * The method is that of M. Akian and S. Detournay, "Multigrid methods for
 * two-player zero-sum stochastic games": find v : X -> R with
 *
 *     v(x) = max_{a in A} min_{b in B} ( sum_y mu p(y|x,a,b) v(y) + r(x,a,b) )
 *
 * (Sec. 2, Eq. (eq1)) by policy iteration (Algorithm 2 with Algorithm 1 as its
 * inner loop, Sec. 4.1-4.2), solving every policy-fixed linear system
 * (I - mu M^{alpha beta}) v = r^{alpha beta} (Eq. (LSPI)) with algebraic
 * multigrid (Sec. 4.3, Algorithm 3; the combination is "AMGpi", Sec. 5.1), and,
 * for Isaacs grids, the full multilevel scheme FAMGpi (Algorithm 4, Sec. 5.2).
 *
 * Conventions for every entry point:
 *  - All pointers are plain host or device pointers.  Data passed in is COPIED
 *    (the caller keeps ownership); data read out is written to the caller's
 *    buffer.  Host buffers may be pageable or pinned; device pointers must be
 *    on the solver's device.  Copies use cudaMemcpyDefault on the solver's
 *    stream, and each call returns only after its work on that stream is done.
 *  - A call that returns anything but GS_OK leaves the solver as it was before
 *    the call, except gamesolve_solve, which keeps the best iterate reached.
 *  - There is no CPU fallback: every step of the method runs in the library's
 *    own CUDA kernels.  A missing or unusable GPU gives GS_ECUDA.
 *  - Not thread-safe per solver; distinct solvers may be used concurrently.
 */
#ifndef GAMESOLVE_H
#define GAMESOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_solver gs_solver;   /* opaque; owns all of its device memory */

typedef enum {
    GS_OK = 0,
    GS_EINVAL = 1,      /* invalid argument or input data (nothing changed) */
    GS_ENOMEM = 2,      /* device memory budget or allocation exceeded */
    GS_ENOTCONV = 3,    /* iteration caps reached; best iterate kept */
    GS_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    GS_ECUDA = 5,       /* CUDA runtime error (message via gamesolve_last_error) */
    GS_ESTATE = 6       /* call out of order (e.g. solve before a problem is set) */
} gs_status;

typedef enum {
    GS_PREC_FP64 = 0,        /* every step in float64 */
    GS_PREC_MIXED = 1,       /* float32 V-cycles inside float64 iterative refinement: the
                                residual, the value update, the coarsest inverse and the
                                stored values in float64; the Galerkin set-up (Isaacs
                                grids) in float32 with every coarse row sum carried by
                                cancellation-free identities, never summed from entries;
                                improvement decisions screened in float32 with a proven
                                margin and a float64 fallback, so they are the float64
                                decisions.  The result meets the same float64 floor. */
    GS_PREC_MIXED_BF16 = 2   /* as MIXED, with the V-cycle's coarse operators and
                                interpolation weights (Isaacs grids) or the transition
                                probabilities of the relaxation (finite games) stored in
                                bfloat16; the arithmetic stays float32 */
} gs_precision;

/* Solver options.  Fill with gamesolve_default_options, then override. */
typedef struct {
    int32_t precision;     /* gs_precision */
    double  eps;           /* policy iteration stops when |F(v) - v|_inf <= eps (Sec. 5.1)
                              or when MAX's policy is unchanged; 0 = the latter only */
    int32_t max_outer;     /* cap on MAX policy iterations (Algorithm 2) */
    int32_t max_inner;     /* cap on MIN policy iterations per MAX step (Algorithm 1) */
    int32_t nu1, nu2;      /* pre/post C/F relaxation sweeps per level (Algorithm 3) */
    int32_t max_cycles;    /* cap on V-cycles (refinement steps) per linear system */
    double  lin_tol;       /* linear solve stops when |b - A v|_inf <= lin_tol * |v|_inf,
                              or when the residual stops decreasing (float64 floor) */
    int32_t coarse_max;    /* coarsest multigrid level has at most this many unknowns */
    int32_t fmg;           /* 1: FAMGpi (Algorithm 4) for Isaacs grids; 0: flat AMGpi */
    int32_t fmg_side;      /* FAMGpi coarsest grid side (2^k - 1), e.g. 31 */
    double  fmg_c;         /* FAMGpi per-level tolerance eps_l = fmg_c * h_l^2 */
    int32_t mu_mode;       /* Isaacs discount: 0 mu = 1/(1+h^2), 1 mu = c0/(c0+h^2) */
    int32_t tail_side;     /* levels of side <= tail_side are relaxed by one thread block,
                              without grid-wide barriers (0 = default, 31) */
    uint64_t mem_budget;   /* bytes of device memory the solver may hold; 0 = no limit */
    void*   stream;        /* cudaStream_t for all work; NULL = the legacy default stream */
    double  pi_rtol;       /* policy evaluations inside the inner loop stop once the residual
                              drops by this factor; before any stopping decision the system is
                              re-solved to the float64 floor and the policies re-checked
                              (0 = every system to the floor) */
    double  setup_reuse;   /* keep the previous Galerkin hierarchy when at most this fraction
                              of the rows of the policy-fixed system changed (0 = always
                              rebuild); the float64 residual test keeps the solution exact */
    int32_t grid_blocks;   /* cap on the thread blocks of one grid-wide launch (0 = the whole
                              GPU); lets solvers on different streams share the GPU */
    int32_t cycle_gamma;   /* coarse-grid visits per level visit (Algorithm 3's gamma): 1 V-cycles
                              (default; 0 reads as 1), 2 W-cycles */
    int32_t nu1_coarse;    /* pre-sweeps on the coarse levels of an Isaacs grid's hierarchy
                              (-1, the default: nu1) */
    int32_t nu2_coarse;    /* post-sweeps on those levels (-1, the default: nu2); the two
                              together must be >= 1 */
    int32_t game_threads;  /* threads per game of a batch of finite games: 256 or 512, or 0
                              (default): 512, autotuned for batches of >= 1024 games (the
                              first solve times both on a sample; the choice is kept for the
                              process per precision, largest game, actions and row length) */
    int32_t cycle_kernel;  /* Isaacs grids' V-cycles: 0 (default) tiled where they apply (each
                              thread block runs a whole smoothing leg of a tile of a level in
                              shared memory, with a halo recomputed by its neighbours: about
                              two grid-wide barriers per level and cycle; the finest level,
                              and coarse levels of side above 511 (255 in float64), keep one
                              phase per colour); 1 one grid-wide phase per
                              relaxation colour.  Same arithmetic per point.  W-cycles always
                              take the latter. */
    int32_t game_solver;   /* policy evaluation of a single finite game (gamesolve_set_game):
                              0 (default) relaxation plus the constant-vector coarse
                              correction (fits random, expander-like games); 1 algebraic
                              multigrid built for every policy-fixed system: strength of
                              connection, C/F splitting, extended+i interpolation, Galerkin
                              coarse operators, V-cycles with C/F Gauss-Seidel (Sec. 4.3; for
                              structured games such as a grid or a chain given as tables).
                              With options.fmg: full multilevel policy iteration on coarse
                              games made by aggregation (Algorithm 4 without a PDE) */
    int32_t amg_coarsening;/* game_solver 1: 0 (default) PMIS independent-set splitting; 1 PMIS
                              followed by the Ruge-Stueben second pass (strong F-F couplings
                              without a common C point promote a point to C); interpolation
                              is extended+i (distance two) with either */
    double  amg_theta;     /* game_solver 1: strength threshold theta (0 = default 0.25) */
} gs_options;

/* Statistics of the last gamesolve_solve (the columns of the paper's tables, Sec. 6). */
typedef struct {
    int32_t outer;          /* k: MAX policy iterations */
    int32_t systems;        /* linear systems solved (sum of #j) */
    int32_t cycles;         /* V-cycles (or refinement steps) over all systems */
    int32_t levels;         /* multigrid levels of the finest hierarchy */
    double  res_inf;        /* |F(v) - v|_inf at the returned v */
    double  res_l2;         /* discrete L2 norm sqrt(mean (F(v) - v)^2) */
    double  seconds;        /* wall time of the solve on the device stream */
    int32_t converged;      /* 1 if a stopping rule was met */
    int32_t fmg_levels;     /* FAMGpi levels run (0 for flat) */
} gs_solve_stats;

/* Fills *opt with the defaults: FP64, eps 0, max_outer 1000, max_inner 1000,
 * V(1,1), max_cycles 200, lin_tol 1e-15, coarse_max 9, flat, fmg_side 31,
 * fmg_c 0.1, literal mu, tail_side 31, no memory budget, default stream,
 * pi_rtol 1e-2, setup_reuse 1e-2, grid_blocks 0, cycle_gamma 1, nu1_coarse and
 * nu2_coarse -1 (as on the finest level), game_threads 0 (autotuned),
 * cycle_kernel 0 (tiled), game_solver 0, amg_coarsening 0,
 * amg_theta 0 (0.25). */
void gamesolve_default_options(gs_options* opt);

/* Creates a solver on the current CUDA device.  opt may be NULL (defaults).
 * Errors: GS_EINVAL (bad option values), GS_ECUDA (no usable device). */
gs_status gamesolve_create(gs_solver** out, const gs_options* opt);

/* Sets a finite game (Sec. 2): n states, m1 MAX actions, m2 MIN actions.
 * Rows of the transition table are indexed (x*m1 + a)*m2 + b; row_ptr has
 * n*m1*m2 + 1 entries (CSR), col[k] in [0, n) and prob[k] = p(col[k] | x, a, b)
 * for k in [row_ptr[row], row_ptr[row+1]); reward has n*m1*m2 entries r(x,a,b).
 * Rows may be substochastic (the missing mass leaves the game), so a row
 * without successors is a "stop" action.
 * A game of at least 4096 states runs on the whole GPU (one cooperative
 * launch: policy iteration on the device with bounded grid barriers); a
 * smaller one runs in one thread block.  Warm starts (set_initial), improve
 * and policy_solve are for Isaacs grids.
 * Errors (GS_EINVAL, solver unchanged): n < 1 or too large, m1 outside
 * [1, 64] or m2 outside [1, 255] (games with more than 8 MAX actions take the
 * float64 improvement without the float32 screen), row_ptr not
 * non-decreasing from 0, a column out of range, a
 * probability outside [0, 1], a row sum above 1 + 1e-12, mu outside (0, 1).
 * mu = 1 (undiscounted, as the stopping games of Sec. 6.2-6.3) is accepted
 * with options.game_solver = 1; every pair of policies must then make the
 * chain leave the state space with probability one (stop rows or
 * substochastic rows reached), else its system is singular and the solve
 * fails. */
gs_status gamesolve_set_game(gs_solver* s, int64_t n, int32_t m1, int32_t m2,
                             const int64_t* row_ptr, const int32_t* col,
                             const double* prob, const double* reward, double mu);

/* Sets a batch of independent finite games (Sec. 2) solved together by one
 * persistent launch: game g has state_offsets[g+1] - state_offsets[g] states
 * (state_offsets has count + 1 entries, starting at 0), m1 and m2 actions for
 * every game, and discount mu[g].  The CSR table concatenates the games' rows
 * in order (game g's row (x*m1 + a)*m2 + b follows all rows of games < g);
 * row_ptr has (total states)*m1*m2 + 1 entries starting at 0; col[k] is a
 * state index within the row's own game.  Values, policies and statistics are
 * read back concatenated in the same state order.  In a batch of two or more
 * games each game must have at most 16384 states (mixed precision) or 8192
 * (float64).  Thread blocks take the games largest first; the first solve of
 * a batch of at least 1024 games picks the block shape (options.game_threads).
 * Errors: as gamesolve_set_game, per row and per game. */
gs_status gamesolve_set_game_batch(gs_solver* s, int32_t count, int32_t m1, int32_t m2,
                                   const int64_t* state_offsets, const int64_t* row_ptr,
                                   const int32_t* col, const double* prob,
                                   const double* reward, const double* mu);

/* Draws a random finite discounted game (Sec. 2) into caller-owned device
 * buffers, on `stream` (NULL = default stream; the call returns once the
 * launch is queued): n states, m1 x m2 action pairs, k successors per row.
 * Row rho = (x*m1 + a)*m2 + b uses outputs rho*17 .. rho*17+16 of the
 * SplitMix64 stream `seed` (Steele, Lea & Flood 2014; a double in [0, 1) is
 * the top 53 bits times 2^-53): outputs 0..k-1 pick k distinct successors
 * uniformly from {0..n-1} (output t gives floor(u (n - t)), stepped past each
 * earlier pick in ascending order), outputs 8..8+k-1 give -log1p(-u) draws
 * normalised to probabilities (pairwise sum for k = 8, left to right
 * otherwise; the last probability set to one minus the others), output 16 the
 * reward 2u - 1.  Successors are stored in increasing column order.
 * row_ptr: n*m1*m2 + 1 int64 (rho*k); col, prob: n*m1*m2*k; reward: n*m1*m2.
 * Errors: GS_EINVAL (n < 1 or >= 2^31, m1 outside [1, 64], m2 outside
 * [1, 255], k outside [1, min(8, n)], a NULL or non-device buffer). */
gs_status gamesolve_random_game(int64_t n, int32_t m1, int32_t m2, int32_t k, uint64_t seed,
                                int64_t* row_ptr, int32_t* col, double* prob, double* reward,
                                void* stream);

/* Sets the random game of gamesolve_random_game (same n, m1, m2, k, seed)
 * with discount mu in (0, 1), drawn on the device: no table crosses the host.
 * Scratch of the table's size is held during the call.
 * Errors: as gamesolve_random_game and gamesolve_set_game. */
gs_status gamesolve_set_random_game(gs_solver* s, int64_t n, int32_t m1, int32_t m2, int32_t k,
                                    uint64_t seed, double mu);

/* Sets the two-sided stopping game on a line of Sec. 6.3 (Eq. (exVI2stop),
 * discretised): states x_1..x_n, n = 2^k - 1 <= 2047 (the interior points of a
 * uniform grid of n + 2 points), end values v_left = v(x_0), v_right =
 * v(x_{n+1}); actions 0 = stop and 1 = continue for both players (m1 = m2 = 2):
 *   F(v; x, a, 0) = psi2[x]   MIN stops (also when both stop),
 *   F(v; x, 0, 1) = psi1[x]   MAX stops alone,
 *   F(v; x, 1, 1) = (v(x-1) + v(x+1)) / 2 + c[x]   both continue (undiscounted,
 *   the central difference of 0.5 v'' with c = h^2 r).
 * c, psi1, psi2: n doubles each, host or device, copied; psi1 <= psi2.
 * gamesolve_solve then runs AMGpi (options.fmg = 0) or FAMGpi from one
 * interior point (options.fmg = 1, eps_l = options.fmg_c h_l^2; a grid twice
 * as coarse takes the stop values at its points and 4 c), entirely on the
 * device in one thread block: every policy-fixed system (tridiagonal) is
 * solved by a one-dimensional algebraic multigrid (C points at odd positions,
 * operator-dependent interpolation, Galerkin coarse operators, C/F
 * relaxation) to the float64 floor.  get_value returns n doubles, get_policy
 * alpha (n) and beta (2n, beta(x, a) at [2x + a]).
 * Errors: GS_EINVAL for n not 2^k - 1 in [1, 2047], a missing array, a value
 * not finite or psi1 > psi2. */
gs_status gamesolve_set_stopping_line(gs_solver* s, int32_t n, const double* c,
                                      const double* psi1, const double* psi2, double v_left,
                                      double v_right);

/* Per-game results of the last solve of a game batch: stats[4g .. 4g+3] =
 * (MAX policy iterations, linear systems, multigrid cycles, converged) and
 * res[g] = |F(v) - v|_inf at the returned value.  Either pointer may be NULL.
 * Errors: GS_ESTATE when no solved batch is held. */
gs_status gamesolve_get_batch_stats(const gs_solver* s, int32_t* stats, double* res);

/* Threads per game the last solve of a game batch ran with (256 or 512; 0 for
 * a single large game run on the whole grid).  Games are taken largest first.
 * Errors: GS_EINVAL (NULL argument), GS_ESTATE when no solved batch is held. */
gs_status gamesolve_get_batch_shape(const gs_solver* s, int32_t* threads);

/* Sets the finite-difference Isaacs game on the unit square (Sec. 3.3, the
 * upwind scheme (decent) with the centred scheme (centre), scaled to the form
 * of Eq. (eq1) as Sec. 6.1 does for Eq. (Iex1d)): side x side interior points,
 * h = 1/(side+1), Dirichlet v = 0 on the boundary, actions a, b in {0..3}
 * indexing the directions +x1, -x1, +x2, -x2, drift (e_a - e_b)/2, one
 * normaliser c0 = 2 + h, reward (1-mu)(sin(pi x1) sin(pi x2) + 0.1(a-b) + xi(x)).
 * variant 0: plain (m1 = m2 = 4).  variant 1: obstacle (Sec. 3.2, Eq. (VI)):
 * MAX also has a = 4, "stop", worth psi(x) = 0.2 - |x - (1/2,1/2)|^2.
 * xi: per-state noise, side*side doubles in row-major order (first
 * coordinate fastest), host or device; NULL draws xi(x) = 0.1 u_x - 0.05 with
 * u_x the x-th double of the SplitMix64 stream `seed`.
 * The multigrid hierarchy coarsens by 2 per level, so side must be 2^k - 1.
 * Errors: GS_EINVAL if side is not 2^k - 1 (1 <= k <= 14), side is below
 * options.fmg_side when options.fmg is set, or variant is not 0 or 1. */
gs_status gamesolve_set_isaacs_grid(gs_solver* s, int32_t side, int32_t variant,
                                    uint64_t seed, const double* xi);

/* Optional warm start for the next solve (Algorithm 4 passes the same three
 * things to AMGpi): v0 (n doubles), alpha0 (n bytes), beta0 (n*m1 bytes,
 * beta(x, a) at [x*m1 + a]).  Any pointer may be NULL: v0 defaults to 0,
 * alpha0 to action 0 (stop everywhere for the obstacle variant), and beta0 to
 * MIN's best reply to v0.  Errors: GS_ESTATE (no problem set), GS_EINVAL
 * (an action out of range). */
gs_status gamesolve_set_initial(gs_solver* s, const double* v0,
                                const uint8_t* alpha0, const uint8_t* beta0);

/* Runs AMGpi (or FAMGpi if options.fmg) from the current initial data.
 * stats may be NULL.  Returns GS_ENOTCONV when a cap was reached (the best
 * iterate is kept and readable): max_outer, or max_cycles in any policy
 * evaluation (an evaluation that stops short of the float64 floor ends the
 * iteration, since no policy decision may rest on it; under FAMGpi the finer
 * levels are then not run).  GS_ESTATE when no problem is set. */
gs_status gamesolve_solve(gs_solver* s, gs_solve_stats* stats);

/* Copies the value v (n doubles) to v_out (host or device). */
gs_status gamesolve_get_value(const gs_solver* s, double* v_out, int64_t n);

/* Copies MAX's policy alpha (n bytes) and MIN's policy beta (n*m1 bytes,
 * beta(x, a) for every a) to the caller's buffers (either may be NULL). */
gs_status gamesolve_get_policy(const gs_solver* s, uint8_t* alpha, uint8_t* beta);

/* One policy improvement (Algorithm 2 step 2 with MIN's reply for every a,
 * Eq. (eq1) and (ILPI)) at the value v (n doubles, host or device) against the
 * current policies (the keep-current tie rule needs them).  Writes
 * alpha' (n bytes), beta' (n*m1 bytes) and F(v) (n doubles); any output may
 * be NULL.  Does not change the solver's policies or value. */
gs_status gamesolve_improve(gs_solver* s, const double* v, uint8_t* alpha_out,
                            uint8_t* beta_out, double* fv_out);

/* Solves the policy-fixed system (I - mu M^{alpha beta}) w = r^{alpha beta}
 * of Eq. (LSPI) for the given policies (alpha: n bytes, beta: n*m1 bytes) with
 * the solver's multigrid method and precision, from the initial guess w0
 * (NULL = 0).  Writes w (n doubles).  stats (may be NULL) gets cycles, the
 * final |b - A w|_inf in res_inf and converged.  Returns GS_ENOTCONV (w
 * holds the last iterate) when options.max_cycles is reached before the
 * float64 floor. */
gs_status gamesolve_policy_solve(gs_solver* s, const uint8_t* alpha, const uint8_t* beta,
                                 const double* w0, double* w_out, gs_solve_stats* stats);

/* The two interpolations of FAMGpi (Algorithm 4, Sec. 5.2) from an Isaacs
 * grid of side side_c to the grid of side 2 side_c + 1 whose points include
 * it (coarse point (P, Q), 1-based, is fine point (2P, 2Q)):
 *  - value interpolation I: a fine point that is a coarse point keeps its
 *    value; any other takes the mean of v over its coarse neighbours N(x) at
 *    distance <= the coarse step, boundary neighbours counting with their
 *    Dirichlet value 0 (2 neighbours on a cell edge, 4 at a cell centre);
 *  - strategy interpolation U: coarse points keep alpha and beta(., a); a new
 *    fine point copies those of the interior member of N(x) with the lowest
 *    row-major index.
 * variant 0 (m1 = 4) or 1 (obstacle, m1 = 5).  Inputs: v_c (n_c doubles),
 * alpha_c (n_c bytes), beta_c (n_c*m1 bytes, beta(x, a) at [x*m1 + a]), n_c =
 * side_c^2; outputs (any may be NULL): v_f, alpha_f, beta_f likewise on the
 * fine grid.  Host or device pointers; the call allocates its own device
 * buffers and runs on `stream` (NULL = legacy default), returning when done.
 * Errors: GS_EINVAL for side_c outside [1, 8191], variant not 0/1, a missing
 * input or an action out of range. */
gs_status gamesolve_fmg_interpolate(int32_t side_c, int32_t variant, const double* v_c,
                                    const uint8_t* alpha_c, const uint8_t* beta_c, double* v_f,
                                    uint8_t* alpha_f, uint8_t* beta_f, void* stream);

/* Iteration counts per level of the last gamesolve_solve of an Isaacs grid
 * (the per-level columns of the paper's FAMGpi tables, Sec. 6): for level k,
 * coarsest first, stats[3k .. 3k+2] = (grid side, MAX policy iterations,
 * linear systems solved).  A flat solve has one level.  At most cap levels
 * are written; *levels (may be NULL) receives the number of levels.
 * Errors: GS_EINVAL (bad arguments), GS_ESTATE (no solved Isaacs grid). */
gs_status gamesolve_get_level_stats(const gs_solver* s, int32_t* stats, int32_t cap,
                                    int32_t* levels);

/* Self-test of the bounded grid-wide barrier (failure detection; the paper has
 * no counterpart).  Every cooperative kernel of the library synchronises its
 * thread blocks with a barrier whose waits give up after a time limit (2 s in
 * the solvers), raise an error flag that releases the other waiters, and make
 * the call return GS_ETIMEOUT instead of hanging the GPU.  This call runs that
 * barrier alone: a cooperative launch of `blocks` blocks (clamped to what can
 * be resident at once) passes it `rounds` times with each wait limited to
 * limit_ns nanoseconds (1e3 .. 1e8).  absent_block in [0, blocks) names a
 * block that returns without ever arriving, so the others' first wait runs out
 * (-1: every block arrives).  *passed (may be NULL) receives the number of
 * barrier passages completed, summed over blocks.  Returns GS_ETIMEOUT when a
 * wait gave up (the context stays usable), GS_OK when every round completed,
 * GS_EINVAL for arguments out of range. */
gs_status gamesolve_selftest_barrier(int32_t blocks, int32_t absent_block, uint64_t limit_ns,
                                     int32_t rounds, void* stream, int32_t* passed);

/* Kernel classes that gamesolve_trace can time (diagnostics). */
typedef enum {
    GS_K_NONE = 0,
    GS_K_IMPROVE = 1,        /* policy improvement fused with the assembly (one launch) */
    GS_K_MG_SETUP = 2,       /* Galerkin set-up of one policy-fixed system (one launch) */
    GS_K_MG_CYCLES = 3       /* V-cycles and the float64 stopping test of one system */
} gs_kernel_class;

/* Selects one kernel class whose launches the following solves bracket with
 * CUDA events on the solver's stream (GS_K_NONE: off) and clears the totals.
 * Costs a few microseconds of host time per bracketed launch. */
gs_status gamesolve_trace(gs_solver* s, int32_t kernel_class);

/* Totals of the traced class since gamesolve_trace: summed device time in
 * milliseconds and number of launches.  Either pointer may be NULL. */
gs_status gamesolve_trace_read(gs_solver* s, double* total_ms, int64_t* launches);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t gamesolve_kernel_launches(void);

/* Allocation-free policy-fixed solve for small Isaacs grids.  The paper has
 * no counterpart: this is a service for callers that cannot let a library
 * allocate device memory (a host whose device memory is all owned by its own
 * caching allocator, a real-time loop that must not pay for cudaMalloc /
 * cudaFree or the device-wide synchronisation they can imply, or code running
 * where CUDA allocation calls are not permitted).
 * It solves the same system as gamesolve_policy_solve, (I - mu M^{alpha beta})
 * w = r^{alpha beta} on the Isaacs game of gamesolve_set_isaacs_grid (side,
 * variant, seed, xi; literal mu), with the default multigrid options and the
 * given precision, and allocates no device memory: its scratch is one
 * 2.5 MiB file-scope device array that every GPU loading the library holds
 * until the process exits.
 *  - side must be 2^k - 1 and at most 127 (GS_EINVAL beyond that).
 *  - alpha (n bytes), beta (n*m1 bytes), w0 (n doubles, NULL = start from 0;
 *    w0 == w is allowed and starts from w's contents), xi (n doubles, NULL =
 *    SplitMix64 stream `seed`) and the output w (n doubles) must be device
 *    memory of the current device, or managed memory (GS_EINVAL otherwise).
 *  - Returns GS_ENOTCONV (w holds the last iterate, stats->converged = 0)
 *    when the default cycle cap is reached before the float64 floor.
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the array and leaves its contents behind; calls that
 *    overlap on the GPU (other streams, other host threads) race on it.
 *  - stream: cudaStream_t for all work (NULL = legacy default stream); the call
 *    returns when its work is done.  stats may be NULL. */
gs_status gamesolve_isaacs_policy_solve_static(int32_t side, int32_t variant, uint64_t seed,
                                               const double* xi, const uint8_t* alpha,
                                               const uint8_t* beta, const double* w0, double* w,
                                               int32_t precision, void* stream,
                                               gs_solve_stats* stats);

/* ---------------------------------------------------------------- serving
 * A request loop around the solvers: requests are queued in arrival order and
 * admitted to worker slots as slots and device memory free up.  Each slot has
 * its own CUDA stream and solver, its grid-wide launches capped to a share of
 * the GPU, so the work of the requests in flight overlaps on the device.
 * Games of fewer than 4096 states (those a solver runs one thread block per
 * game) that wait together with the same kind and action counts are taken by
 * one slot as a batch of up to 256 and solved by one persistent launch
 * (gamesolve_set_game_batch); they share t_start and t_end.  A request's
 * multigrid hierarchy and policies stay on the device for its whole policy
 * iteration; its value and policies are copied to host memory when it
 * completes.  Results do not depend on what else is in flight (the kernels'
 * arithmetic does not depend on timing or on a game's batch; only the number
 * of blocks a grid-wide game reduction uses can change its rounding). */
typedef struct gs_server gs_server;

typedef struct {
    int32_t kind;            /* 1 Isaacs grid, 2 finite game given as a table, 3 random finite
                                game given by its seed (gamesolve_set_random_game) */
    int32_t side;            /* Isaacs: grid side (2^k - 1) */
    int32_t variant;         /* Isaacs: 0 plain, 1 obstacle */
    int32_t m1, m2;          /* games: actions */
    uint64_t seed;           /* Isaacs: noise stream; random game: its stream */
    int64_t n;               /* games: states */
    const int64_t* row_ptr;  /* game: CSR table as for gamesolve_set_game (copied at submit) */
    const int32_t* col;
    const double* prob;
    const double* reward;
    double mu;               /* games: discount */
    int32_t flags;           /* GS_REQ_BORROW: the table is not copied at submit; the caller
                                keeps it valid (host or device memory) until the request is done */
    int32_t k;               /* random game: successors per row, 1..8 (0 = 8) */
} gs_request;

enum { GS_REQ_BORROW = 1 };

typedef struct {
    int32_t state;           /* 0 queued, 1 running, 2 done */
    int32_t status;          /* gs_status of the solve, once done */
    double t_submit, t_start, t_end;   /* seconds since the server was created */
    int64_t n;               /* states of the request */
    gs_solve_stats stats;    /* statistics of its solve */
} gs_ticket_info;

/* Starts `slots` worker threads on the current device, each creating a solver
 * with `opt` (NULL = defaults) on its own stream.  Unless opt->grid_blocks is
 * set, a slot's grid-wide launches are capped at 2 x (SMs) / slots blocks; on
 * a mixed stream of Isaacs grids and large games 2 slots served the most
 * requests per second (whole-GPU launches, one request's host steps hidden
 * behind the other's kernels).  mem_budget: device bytes the
 * requests in flight may hold together (0 = half the free memory); a request
 * larger than the budget runs when nothing else is in flight.
 * Errors: GS_EINVAL (slots outside [1, 64] or bad options), GS_ECUDA. */
gs_status gamesolve_server_create(gs_server** out, const gs_options* opt, int32_t slots,
                                  uint64_t mem_budget);

/* Queues a request; its data is copied before the call returns unless the
 * request borrows it (GS_REQ_BORROW).  *ticket
 * identifies it.  Errors: GS_EINVAL (invalid request).  Table errors found
 * when it runs are reported in its ticket's status. */
gs_status gamesolve_server_submit(gs_server* srv, const gs_request* req, int64_t* ticket);

/* State of a request without waiting (GS_EINVAL for an unknown ticket). */
gs_status gamesolve_server_poll(gs_server* srv, int64_t ticket, gs_ticket_info* info);

/* Waits until the request is done, then fills *info (may be NULL). */
gs_status gamesolve_server_wait(gs_server* srv, int64_t ticket, gs_ticket_info* info);

/* Copies a done request's value (n doubles) and policies (n bytes, n*m1
 * bytes; any pointer may be NULL) and forgets the ticket.  Returns the
 * request's solve status; GS_ESTATE if it is not done yet. */
gs_status gamesolve_server_result(gs_server* srv, int64_t ticket, double* v_out, int64_t n,
                                  uint8_t* alpha, uint8_t* beta);

/* Stops the workers after the requests in flight finish; queued requests
 * that have not started are dropped.  NULL is a no-op. */
void gamesolve_server_destroy(gs_server* srv);

/* Frees the solver and all of its device memory.  NULL is a no-op. */
void gamesolve_destroy(gs_solver* s);

/* Static description of a status code. */
const char* gamesolve_strerror(gs_status st);

/* Text of the last error raised on this thread (CUDA or validation detail). */
const char* gamesolve_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GAMESOLVE_H */
