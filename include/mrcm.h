/*
 * mrcm.h - C ABI of libmrcm, the GB300 (sm_103a) implementation of the
 * Multiscale Robin Coupled Method (MRCM) pressure solve for 3-D single-phase
 * Darcy flow (arXiv 2103.08513).
 *
 * The library runs the paper's Alg. MRCM on one GPU:
 *   mrcm_factor_local       Alg. MRCM first loop, "Assembly": local TPFA +
 *                           Robin matrices A^H_l (Eq. aijk, Eq. localomegapar,
 *                           Eq. localomegaint) and their factorisation
 *   mrcm_solve_mbf          Alg. MRCM first loop, "LocalSolver": all MBFs and
 *                           particular solutions (Eq. multiscale_functions,
 *                           Eq. particular_problem_discrete) and their traces
 *   mrcm_assemble_interface Alg. MRCM "Assembly" of Eq. interface_problem
 *                           (Eq. sec2-int-APP, Eq. sec2-int-AUU, Eq. sec2-int-bU)
 *   mrcm_solve_interface    Alg. MRCM "InterfaceSolver"
 *   mrcm_reconstruct        Alg. MRCM second loop, "ReconstructMscSolution"
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: nx x ny x nz cells of size hx x hy x hz; cell c = i + nx*(j + ny*k)
 * (x fastest).  Subdomains are the Cartesian products of per-axis edge lists;
 * subdomain l = ix + Nx*(iy + Ny*iz).  The lower-indexed side of every
 * interface is the side with the lower coordinate, so n_hat is the +axis.
 *
 * Interface space V_H: on every interface normal to axis a, fine faces are
 * grouped in patches of patch[a][0] x patch[a][1] faces along the two
 * tangential axes taken in increasing axis order (0 = whole face), tiled from
 * the lower corner, the last patch truncated.  Basis functions are numbered by
 * normal axis, then lower subdomain, then patch (second tangential axis slow).
 * Interface unknowns X = (pi^p_0..pi^p_{NV-1}, pi^u_0..pi^u_{NV-1}).
 *
 * Pointers: "device" pointers must be CUDA device (or managed) memory on the
 * device that is current when the call is made; the library never frees
 * caller memory.  The workspace `ws` (size from mrcm_query_workspace, 256-byte
 * aligned) is owned by the caller and must stay the same buffer for all calls
 * of one solve.  The handle owns only its host tables and a device copy of
 * them, allocated on the first device call (which synchronises the stream
 * once; make that call before any stream capture).
 *
 * Streams: every device call is asynchronous on `stream` (a cudaStream_t; NULL
 * is the legacy default stream).  Calls on one handle must not overlap.
 *
 * Errors: every call returns an mrcm_status; mrcm_last_error() describes the
 * last failure of a handle.  No call aborts, traps or falls back to the CPU.
 */
#ifndef MRCM_H
#define MRCM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MRCM_OK = 0,
    MRCM_ERR_INVALID_ARG = 1,       /* bad config, pointer or size */
    MRCM_ERR_CUDA = 2,              /* a CUDA runtime call failed */
    MRCM_ERR_NOT_SPD = 3,           /* a local block pivot was not positive */
    MRCM_ERR_NO_CONVERGENCE = 4,    /* iterative refinement did not reach its tolerance */
    MRCM_ERR_SINGULAR_INTERFACE = 5,/* zero pivot in the interface factorisation */
    MRCM_ERR_TIMEOUT = 6,           /* a bounded device wait gave up */
    MRCM_ERR_OOM = 7,               /* workspace too small */
    MRCM_ERR_NOT_IMPLEMENTED = 8,   /* option not supported by this build */
    MRCM_ERR_STATE = 9              /* calls made out of order */
} mrcm_status;

enum { MRCM_BETA_CONST = 0, MRCM_BETA_ALPHA_H_OVER_K = 1 };
enum { MRCM_BC_NOFLOW = 0, MRCM_BC_DIRICHLET = 1 };
enum {
    MRCM_FP64 = 0,          /* local factor and solves in FP64 (one FP64 refinement step) */
    MRCM_FP32_IR = 1,       /* FP32 factor/solves + FP64 iterative refinement */
    MRCM_TF32_IR = 2,       /* tensor-core TF32 solves + FP64 iterative refinement */
    MRCM_LEARNED_PCG = 3    /* learned form: MBFs by warm-started FP32 CG inside FP64 refinement
                               (mrcm_solve_mbf_learned), FP64 direct fallback */
};

/* Problem description (Sec. "Domain decomposition and Darcy solvers").
 *  nx, ny, nz         cells per axis (>= 1)
 *  hx, hy, hz         cell sizes (> 0)
 *  n_cuts[a], cuts[a] per-axis subdomain edge list (host pointer, n_cuts[a]
 *                     positive ints summing to the axis' cell count); read
 *                     during mrcm_setup only
 *  patch[a][0..1]     patch size in faces on faces normal to axis a, along
 *                     the first/second tangential axis (0 = whole face)
 *  beta_mode          MRCM_BETA_CONST (beta = beta_const) or
 *                     MRCM_BETA_ALPHA_H_OVER_K (Eq. Robin_par: beta = alpha *
 *                     H_a / K_a with H_a the subdomain edge along the normal
 *                     and K_a the normal permeability of the adjacent cell of
 *                     the side being solved)
 *  bc_type[a][side]   wall condition on the low (side 0) / high (side 1) wall
 *                     normal to axis a: MRCM_BC_NOFLOW or MRCM_BC_DIRICHLET
 *  bc_value[a][side]  Dirichlet pressure of that wall
 *  precision          MRCM_FP64 / MRCM_FP32_IR / MRCM_TF32_IR
 *  ir_max_sweeps      refinement sweeps after the first solve (mixed modes;
 *                     MRCM_FP64 always takes one)
 *  ir_tol             per-column stop: ||r||_2 <= ir_tol * ||b||_2
 *  wave_bytes         memory budget (bytes) of the local block factors: when
 *                     positive, subdomains are processed in waves whose
 *                     factors fit the budget (the factors of one wave are
 *                     dropped before the next is factored); 0 = one wave
 *  tune_cache         path of the autotuner cache (text), or NULL; read at
 *                     the first device call, written by mrcm_autotune
 *  interface_refine   FP64 refinement steps of the interface solve after the
 *                     LDL^T solve: 0 = default (1), -1 = none, k > 0 = k
 *  fallback_cap       mixed modes: subdomains whose columns are still above
 *                     ir_tol after ir_max_sweeps are factored and solved again
 *                     in FP64 (the direct fallback), at most this many per
 *                     wave (their FP64 block factors take a workspace region
 *                     of that many slots); 0 = default max(16, n_sub / 64)
 *                     (at most n_sub), -1 = no fallback.  Subdomains beyond
 *                     the cap, or with slab blocks above 224 (the FP64 factor's
 *                     limit), stay unconverged and are counted by
 *                     mrcm_read_status */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int n_cuts[3];
    const int* cuts[3];
    int patch[3][2];
    int beta_mode;
    double alpha, beta_const;
    int bc_type[3][2];
    double bc_value[3][2];
    int precision;
    int ir_max_sweeps;
    double ir_tol;
    size_t wave_bytes;
    const char* tune_cache;
    int interface_refine;
    int fallback_cap;
} mrcm_config;

/* Sizes derived by mrcm_setup (host-side; no GPU needed). */
typedef struct {
    long long n_cells;          /* nx*ny*nz */
    int n_sub;                  /* subdomains */
    int n_basis;                /* NV, basis functions of V_H */
    long long n_faces;          /* Robin faces counted once per side */
    int max_rhs;                /* max over l of m_l = 2|I^l| + 1 */
    long long total_rhs;        /* sum over l of m_l */
    long long nnz_interface;    /* nonzeros of A^int in the CSR pattern */
    int n_fronts;               /* internal nodes of the interface elimination tree */
    int max_front;              /* largest dense front */
    double front_flops;         /* flops of an LU of the same fronts (2x the LDL^T) */
    double local_factor_flops;  /* sum of N_l b_l^2: band-Cholesky flops of the local factors */
    double local_solve_flops;   /* flops of one solve sweep over all MBF columns */
    int max_block;              /* largest slab block size b */
    long long mbf_entries;      /* sum over l of m_l * N_l (MBF array length) */
    double ldl_flops;           /* flops of the interface LDL^T (lower triangle) */
    double ldl_update_flops;    /* part of ldl_flops in the trailing (Schur) updates */
    int n_waves;                /* memory-bounded waves of the local phase */
    int max_front_ne;           /* largest eliminated block of a front (its substitutions
                                   run on a cluster of CTAs from 128 on) */
    int max_front_nb;           /* largest boundary block of a front (its back substitution
                                   is split into row chunks above 128) */
    double ldl_update_tensor_flops; /* BF16 tensor-core flops the emulated trailing updates
                                   execute (all slice products of the steps that emulate;
                                   ldl_update_flops counts the FP64 work they stand for) */
} mrcm_sizes;

typedef struct mrcm_handle mrcm_handle;

/* Validate `cfg`, build the decomposition, interface-space, face and
 * elimination-tree tables on the host.  Returns INVALID_ARG for inconsistent
 * edge lists, non-positive sizes, unsupported block sizes, or a problem whose
 * pressure is undetermined (one subdomain and no Dirichlet wall).  On success
 * *out owns the tables; release with mrcm_destroy.  No device work. */
mrcm_status mrcm_setup(const mrcm_config* cfg, mrcm_handle** out);

/* Workspace bytes for one solve and the interface unknown count 2*NV. */
mrcm_status mrcm_query_workspace(const mrcm_handle* h, size_t* ws_bytes, size_t* n_interface_unknowns);

/* Derived sizes (see mrcm_sizes). */
mrcm_status mrcm_query_sizes(const mrcm_handle* h, mrcm_sizes* out);

/* Algorithmic cost of the paper's local solver (host only): the flops of a
 * sparse direct LDL^T of every subdomain's local matrix under exact minimum
 * degree ordering (ties: lowest box-lexicographic cell index; the stand-in for
 * the paper's AMD ordering, Sec. "MBFs: LocalSolver()"), column j costing
 * c_j (c_j + 3) for its c_j below-diagonal entries, and of solving all m_l
 * right-hand sides once with it (4 nnz(L) m_l).  Subdomains above 4096
 * cells: NOT_IMPLEMENTED.  Computed once per box shape per call. */
mrcm_status mrcm_query_local_ldl(const mrcm_handle* h, double* factor_flops, double* solve_flops);

/* Basis function i of V_H: normal axis, lower/upper subdomain, fine faces. */
mrcm_status mrcm_query_basis(const mrcm_handle* h, int i, int* axis, int* sub_lo, int* sub_hi, int* n_faces);

/* Assemble every local matrix A^H_l from K and factor it (with several
 * memory-bounded waves the factorisation moves to mrcm_solve_mbf, wave by
 * wave).
 *  K   device, FP64 [3][nz][ny][nx] (Kxx, Kyy, Kzz), all entries > 0 and finite
 *  ws  device workspace, ws_bytes >= mrcm_query_workspace
 * The local matrices are built in FP64 (Eq. aijk with harmonic means; Robin
 * faces with T_R = A_f / (h_n/(2K_n) + beta)); the block factor is kept in
 * FP64 or FP32 by cfg.precision.  Non-positive pivots are reported as
 * MRCM_ERR_NOT_SPD by the next synchronising call (mrcm_solve_mbf's status
 * read-back) rather than here. */
mrcm_status mrcm_factor_local(mrcm_handle* h, const double* K, void* ws, size_t ws_bytes, void* stream);

/* Solve all MBF and particular right-hand sides of every subdomain (FP64, or
 * low precision + FP64 iterative refinement) and reduce the flux traces to
 * the per-subdomain interface blocks.
 *  f   device, FP64 [nz][ny][nx] source density (div u = f) */
mrcm_status mrcm_solve_mbf(mrcm_handle* h, const double* f, void* ws, void* stream);

/* Gather the per-subdomain blocks into A^int (CSR, FP64) and b^int, then
 * factor the interface system: J A^int (J = diag(I, -I)) is symmetric
 * quasi-definite, so it is scaled symmetrically and factored by a nested-
 * dissection multifrontal LDL^T without pivoting (FP64).  When no wall is
 * Dirichlet the pressure constant is removed by adding -|A_00| e_0 e_0^T,
 * which yields the solution with pi^p_0 = 0.  A zero pivot is reported as
 * MRCM_ERR_SINGULAR_INTERFACE by mrcm_read_status. */
mrcm_status mrcm_assemble_interface(mrcm_handle* h, void* ws, void* stream);

/* Solve the interface system with the factor of mrcm_assemble_interface and
 * two FP64 iterative-refinement steps (CSR residuals).
 *  X   device, FP64 [2*NV], output */
mrcm_status mrcm_solve_interface(mrcm_handle* h, double* X, void* ws, void* stream);

/* Reconstruct p and u from the MBFs and X (reconstruction option 1).
 *  X      device FP64 [2*NV] (input)
 *  p      device FP64 [nz][ny][nx] (output); shifted to zero mean when no wall
 *         is Dirichlet
 *  u      device FP64 [6][nz][ny][nx] (output): +axis velocity on the
 *         x-low, x-high, y-low, y-high, z-low, z-high face of each cell, as
 *         seen from the cell's own subdomain (two values on Gamma faces)
 *  mass_residual_max  device FP64 [1] (output): max over cells of
 *         |sum of outward fluxes - f V|; may be NULL */
mrcm_status mrcm_reconstruct(mrcm_handle* h, const double* X, double* p, double* u,
                             double* mass_residual_max, void* ws, void* stream);

/* Mean velocity post-processing (Eq. locprob_submean; the "Mean" method of
 * the paper's two-phase section), for a transport step that needs a velocity
 * conservative on the fine grid.  On every fine Gamma face the two sides'
 * velocities of `u` are averaged, Ubar = (u+ + u-)/2; every subdomain then
 * re-solves its TPFA problem (Eq. aijk, harmonic means) with Neumann data:
 * Ubar.n on its Gamma faces and u.n on the domain walls.  The pure Neumann
 * matrix is factored and solved like the local problems (cfg.precision;
 * mixed precision: FP32 block factors, the FP32 solve and up to ten FP64
 * refinement sweeps to a normwise backward error of 1e-13 for every
 * subdomain, then FP64 block factors, in waves inside the factor region, and
 * the FP64 solve with three FP64 refinement steps for the subdomains whose
 * column stayed above it -- their count is what mrcm_read_fallback reports
 * after this call); the
 * subdomain's pressure constant is fixed internally (it does not affect the
 * velocity).
 *  u      device FP64 [6][nz][ny][nx]: the multiscale velocity as written by
 *         mrcm_reconstruct (input)
 *  u_out  device FP64 [6][nz][ny][nx] (output, must not overlap u): TPFA of the
 *         new pressure on interior faces, Ubar on Gamma faces (one value, both
 *         sides), u on walls
 *  mass_residual_max  device FP64 [1] (output, may be NULL): max over cells of
 *         |sum of outward fluxes of u_out - f V|
 * Needs a completed solve (after mrcm_reconstruct or mrcm_solve); it
 * overwrites the local coefficients, factors and MBF columns, so the next
 * solve must start again from mrcm_factor_local (MRCM_ERR_STATE otherwise).
 * The refinement stops on the normwise backward error,
 * ||r|| <= cfg.ir_tol || |b| + |A||x| || (1e-14 when ir_tol is 0); columns that
 * miss it after the three steps are reported by mrcm_read_status. */
mrcm_status mrcm_postprocess_velocity(mrcm_handle* h, const double* u, double* u_out, double* mass_residual_max,
                                      void* ws, void* stream);

/* Two-phase IMPES with a skipping constant (Alg. overview-code; Sec. "The
 * fine grid transport solver", Eq. transporte_discreto, Eq. CFL).  Water
 * saturation S (time rescaled by the porosity), total mobility
 * lambda(S) = S^2/mu_w + (1-S)^2/mu_o, fractional flow
 * phi(S) = M S^2 / (M S^2 + (1-S)^2), M = mu_o/mu_w.  For n_steps steps:
 * every C steps (the first included) K_eff = lambda(S) K is formed, the MRCM
 * pressure solve runs on it (mrcm_solve, not graph-captured) and its velocity
 * is post-processed (mrcm_postprocess_velocity), the time step is
 * dt = cfl min(h) / (phi'_max max|u|) (phi'_max = max of phi' over
 * S = k/1000); then the explicit upwind step
 *   S_c += -(dt/V) sum_faces (phi_upwind - phi(S_c)) q_out + dt max(f_c,0) (1 - phi(S_c))
 * (injectors bring water, producers take the local mixture; walls no-flow).
 *  K      device FP64 [3][nz][ny][nx] absolute permeability
 *  f      device FP64 [nz][ny][nx] source density (sums to zero)
 *  S      device FP64 [nz][ny][nx] saturation, in: S at t = 0, out: after n_steps
 *  t_out  device FP64 [1] (output, may be NULL): the simulated time
 *  tws    device transport workspace of mrcm_transport_query bytes (K_eff,
 *         the solve's p, u, X, the post-processed u, a second S)
 * NOT_IMPLEMENTED with Dirichlet walls.  The last post-processing leaves the
 * handle needing mrcm_factor_local (see mrcm_postprocess_velocity). */
mrcm_status mrcm_transport_query(const mrcm_handle* h, size_t* tws_bytes);
mrcm_status mrcm_impes(mrcm_handle* h, const double* K, const double* f, double* S, double mu_w, double mu_o,
                       double cfl, int C, int n_steps, double* t_out, void* tws, size_t tws_bytes, void* ws,
                       size_t ws_bytes, void* stream);

/* The whole pressure solve: mrcm_factor_local, mrcm_solve_mbf,
 * mrcm_assemble_interface, mrcm_solve_interface and mrcm_reconstruct in
 * order (arguments as there).  With flags & MRCM_SOLVE_GRAPH the sequence is
 * captured into a CUDA graph on the first call (stream must not be NULL; the
 * library's one-time device set-up runs before the capture) and replayed by
 * later calls with the same pointers, workspace size and stream; changing any
 * of them re-captures. */
enum { MRCM_SOLVE_GRAPH = 1 };
mrcm_status mrcm_solve(mrcm_handle* h, const double* K, const double* f, double* X, double* p, double* u,
                       double* mass_residual_max, void* ws, size_t ws_bytes, void* stream, int flags);

/* mrcm_solve with HOST buffers (same layouts): K and f are copied to device
 * staging buffers (allocated by the first call, 11 n_cells + 2 N_V + 1
 * doubles, freed by mrcm_destroy), the solve runs, and X, p, u and
 * mass_residual_max (may be NULL) are copied back, all ordered on `stream`
 * (required, not NULL; the larger copies are split with a library-owned side
 * stream so that two copies run at once).  The results are in the host
 * buffers once `stream` has completed.  With MRCM_SOLVE_GRAPH copies and solve
 * are captured into one CUDA graph (host buffers must then be page-locked)
 * and replayed by later calls with the same pointers, workspace size and
 * stream. */
mrcm_status mrcm_solve_host(mrcm_handle* h, const double* K, const double* f, double* X, double* p, double* u,
                            double* mass_residual_max, void* ws, size_t ws_bytes, void* stream, int flags);

/* Autotuner (run after mrcm_factor_local): times every variant of the local
 * solve kernels (128, 256 or 512 threads per CTA x SIMT block products with
 * 1, 2 or 4 rows per thread, 2 adjacent rows per thread (even blocks) or
 * 3xTF32 tensor-core block products) on
 * this problem, keeps the fastest first-solve and refinement-sweep variants
 * for the handle, and appends them to cfg.tune_cache when one was given (a
 * later mrcm_setup with the same cache and problem shape reuses them without
 * tuning).  Overwrites the MBF array: call mrcm_solve_mbf afterwards. */
mrcm_status mrcm_autotune(mrcm_handle* h, const double* f, void* ws, void* stream, int* solve_variant,
                          int* sweep_variant);

/* Median times (ms) of every local-solve variant in the last mrcm_autotune
 * of this handle (host only): solve_ms[v] the first solve, sweep_ms[v] the
 * cfg.ir_max_sweeps refinement sweeps in one launch (-1 where not timed: FP64
 * handles time no sweeps), and the resident CTAs per SM of each
 * (solve_ctas[v], sweep_ctas[v]).  Writes min(*n, cap) entries of each
 * non-NULL array; *n = the number of variants (0 before any autotune).
 * *sweeps_separate = 1 when the handle runs one launch per sweep (the
 * autotuner measured that faster than one launch for all sweeps), and
 * *sweeps_separate_ms that time for the chosen sweep variant (-1: not timed).
 * Any output pointer may be NULL. */
mrcm_status mrcm_read_tuning_times(const mrcm_handle* h, float* solve_ms, float* sweep_ms, int* solve_ctas,
                                   int* sweep_ctas, int cap, int* n, int* sweeps_separate,
                                   float* sweeps_separate_ms);

/* The kernel variants the handle uses (host only; after mrcm_autotune or a
 * tune-cache hit, else the defaults): local solve first pass and refinement
 * sweep (0-11), factor for blocks with b <= 64 (0 a row per thread, 1 8x8
 * register tiles, 2 4x4 tiles) and for 64 < b <= 128 (0 register tiles,
 * 1 tensor cores with the block in tensor memory).  Any pointer may be NULL. */
mrcm_status mrcm_query_tuning(const mrcm_handle* h, int* solve_variant, int* sweep_variant, int* factor_small,
                              int* factor_mid);

/* Device-side status of the last solve, read back synchronously: number of
 * non-positive local pivots, unconverged refinement columns, interface zero
 * pivots and the refinement sweeps used. */
mrcm_status mrcm_read_status(mrcm_handle* h, void* ws, int* not_spd, int* unconverged,
                             int* interface_zero_pivots, int* sweeps_used);

/* FP64 fallback of the last solve, read back synchronously: subdomains that
 * were re-solved in FP64 after the mixed refinement left columns above
 * ir_tol, and subdomains that needed it but could not have it (over the
 * cap, or slab block above 224); the latter's columns count as unconverged. */
mrcm_status mrcm_read_fallback(mrcm_handle* h, void* ws, int* fallback_subdomains, int* not_recovered);

/* Work counters of the last solve, read back synchronously: MBF entries
 * (cell x right-hand side) swept by the FP64-residual refinement sweeps, summed
 * over sweeps (converged columns drop out of later sweeps). */
mrcm_status mrcm_read_work(mrcm_handle* h, void* ws, long long* swept_entries);

/* Copy device-resident intermediate results for inspection (device -> host,
 * synchronous).  what: 0 = A^int CSR values (nnz_interface doubles), 1 = b^int
 * (2*NV doubles), 2 = CSR row pointers (2*NV+1 ints), 3 = CSR column indices
 * (nnz ints), 4 = MBF columns of subdomain `sub` (m_l x N_l doubles, column
 * k over the subdomain's cells in global-lexicographic order). */
mrcm_status mrcm_export(mrcm_handle* h, void* ws, int what, int sub, void* host_dst, size_t bytes);

/* Per-kernel timing.  enable != 0 records a CUDA event pair on the launching
 * stream around every kernel the library launches from now on (and clears
 * earlier records); enable == 0 stops recording.  Launches are counted
 * whether or not recording is on. */
mrcm_status mrcm_profile(mrcm_handle* h, int enable);

/* Synchronise on the last recorded event and write one line per kernel,
 * "name launches total_ms\n", into buf (host, len bytes, NUL-terminated);
 * *launches (may be NULL) receives the launch count.  Clears the records and
 * the count.  INVALID_ARG if buf is too small (the text is truncated). */
mrcm_status mrcm_profile_report(mrcm_handle* h, char* buf, size_t len, long long* launches);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (2 flops per
 * FMA), the denominator of the library's FP64 roofline fractions (no
 * counterpart in the paper).  Runs a short kernel of independent FMA chains
 * on every SM on `stream` and synchronises it; *tflops (host) receives the
 * best of three timed launches. */
mrcm_status mrcm_measure_fp64_peak(void* stream, double* tflops);

/* Allocation-free local solve of one box subdomain (the paper has no
 * counterpart: this is a deployment variant of the local factor and solve).
 * It is for callers that cannot allocate device memory -- code whose host
 * application owns every device allocation through its own pool, plug-ins
 * that may only touch the buffers handed to them, or real-time loops where a
 * cudaMalloc would stall the device.  It needs no workspace and no handle:
 * its scratch is a fixed 2.26 MB __device__ array inside the library, held by
 * every GPU that loads the library until the process exits.
 *
 * Solves the TPFA problem of Eq. localomegaint / Eq. localomegapar on a box of
 * box[0] x box[1] x box[2] cells of size h (FP64, the same discretisation as
 * mrcm_factor_local / mrcm_solve_mbf): for every cell
 *   sum_interior T (p_c - p_nb) + sum_Robin T_R (p_c - g) + sum_Dirichlet T_D (p_c - g) = f V.
 *  side_type[6]  host; sides x-lo, x-hi, y-lo, y-hi, z-lo, z-hi:
 *                0 no-flow, 1 Robin (-beta u.n + p = g), 2 Dirichlet (p = g)
 *  K     device FP64 [3][box z][box y][box x];  f device FP64 [z][y][x]
 *  g, beta  device FP64, one value per boundary face: side by side in the
 *        order above, each side's faces with its first tangential axis (lower
 *        axis index) fastest; beta is read on Robin sides only
 *  p     device FP64 [z][y][x] output
 *  q_out device FP64, same layout as g: outward integrated flux T (p_c - g)
 *        on Robin and Dirichlet faces, 0 on no-flow faces
 *  not_spd  device int output: 1 if a block pivot was not positive
 * Limits (the fixed scratch): at most 4096 cells, slab block (product of the
 * two shorter edges) <= 128, longest edge x block^2 <= 262144; larger boxes
 * return MRCM_ERR_OOM.  At least one side must be Robin or Dirichlet
 * (MRCM_ERR_INVALID_ARG otherwise).  The first call on a device looks up the
 * scratch address and sets the kernel's shared-memory limit; make that first
 * call before any stream capture.  The looked-up address is kept for the
 * life of the process; calling this entry point again after cudaDeviceReset
 * is not supported.  Every call on a device shares the one
 * scratch array (nothing in it is read before the same call writes it), so
 * calls that overlap on the GPU (different streams, or host threads) race:
 * serialise them. */
mrcm_status mrcm_box_solve_noalloc(const int box[3], const double h[3], const int side_type[6],
                                   const double* K, const double* f, const double* g, const double* beta,
                                   double* p, double* q_out, int* not_spd, void* stream);

/* ---- Learned warm start (no counterpart in the paper) -------------------
 * A small 3-D convolutional network (layers-1 hidden layers of `hidden`
 * channels, 3x3x3 'same' convolutions, leaky ReLU (slope 1/100), logistic output) maps a
 * subdomain's fields to a guess of one P-MBF, which seeds an FP32 conjugate-
 * gradient solve of the local system.  Weights are FP32 (master, Adam
 * moments) and used as BF16 by the convolutions; accumulation is FP32.
 * Tensors are [batch][channel][D][H][W] FP32 device arrays (W fastest).
 * The caller owns every buffer: `state` (mrcm_net_query's state_floats) holds
 * master weights, Adam moments and the BF16 copy; `ws` (ws_bytes for the
 * batch) holds activations and gradients. */
typedef struct mrcm_net mrcm_net;

/* Describe a network for D x H x W boxes (S = D*H*W <= 4096); in_channels
 * and hidden <= 32, 2 <= layers <= 16.  Host only. */
mrcm_status mrcm_net_create(int in_channels, int hidden, int layers, int D, int H, int W, mrcm_net** out);
mrcm_status mrcm_net_query(const mrcm_net* net, int batch, size_t* params, size_t* state_floats,
                           size_t* ws_bytes);
/* He-normal weights from a counter-based generator (splitmix64; the output
 * layer's scaled by 1/10), zero biases and Adam moments.  Synchronises the
 * stream. */
mrcm_status mrcm_net_init(mrcm_net* net, float* state, unsigned long long seed, void* stream);
/* Refresh the BF16 copy after the caller wrote master weights. */
mrcm_status mrcm_net_sync_weights(mrcm_net* net, float* state, void* stream);
/* y[batch][1][D][H][W] = net(x[batch][in][D][H][W]). */
mrcm_status mrcm_net_forward(mrcm_net* net, const float* state, const float* x, float* y, int batch, void* ws,
                             void* stream);
/* Loss against target[batch][1][D][H][W] (*loss, device) and its gradient
 * with respect to the parameters (grad[params], device).  weight NULL: the
 * pressure MSE, mean((y - t)^2).  weight[batch][1][D][H][W] (device, from
 * mrcm_net_flux_weights): the face-flux term is added, mean((1 + w)(y - t)^2)
 * with w = sum of T_R^2 over the cell's Robin faces, T_R (y - t) being the
 * error of the outward flux through such a face. */
mrcm_status mrcm_net_gradient(mrcm_net* net, const float* state, const float* x, const float* target,
                              const float* weight, int batch, float* grad, float* loss, void* ws, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step counts from 1) on the
 * loss of mrcm_net_gradient. */
mrcm_status mrcm_net_train_step(mrcm_net* net, float* state, const float* x, const float* target,
                                const float* weight, int batch, float lr, int step, float* loss, void* ws,
                                void* stream);
void mrcm_net_destroy(mrcm_net* net);

/* Training samples from the method itself (after mrcm_solve_mbf): sample s
 * is P-MBF column c of subdomain l, for the subdomains whose box is the
 * network's W x H x D, enumerated by subdomain then c.  x[s] has 4 channels:
 * log(Kx)/4, log(Kz)/4, the cells next to the faces of basis c (1, else 0) and the
 * cells next to any Robin face; target[s] is the FP64 column rounded to FP32.
 * *n_samples = min(available, max_samples); x/target may be NULL to count.
 * Inputs alone (target NULL) need only mrcm_factor_local; targets need the
 * MBFs (after mrcm_solve_mbf).
 * The first call per box shape uploads a small sample table owned by the
 * handle. */
mrcm_status mrcm_net_samples(mrcm_handle* h, const mrcm_net* net, void* ws, float* x, float* target,
                             int max_samples, int* n_samples, void* stream);

/* The loss weights of the face-flux term for the same samples (after
 * mrcm_factor_local): weight[s][cell] = sum of T_R^2 over the cell's Robin
 * faces (0 for cells without one), [s][D][H][W] FP32 device, the first
 * min(max_samples, available) samples. */
mrcm_status mrcm_net_flux_weights(mrcm_handle* h, const mrcm_net* net, void* ws, float* weight, int max_samples,
                                  void* stream);

/* The learned form of mrcm_solve_mbf, for a handle set up with precision
 * MRCM_LEARNED_PCG (after mrcm_factor_local, which then assembles the local
 * coefficients without factoring).  Every MBF and particular column of every
 * subdomain (Eq. multiscale_functions, Eq. particular_problem_discrete) is
 * solved by FP64 iterative refinement: r = b - A x in FP64, the correction
 * from FP32 conjugate gradients on the Jacobi-scaled local system (to a
 * relative residual of 1e-4, at most cg_maxit iterations), x += correction,
 * at most max_outer corrections, until ||r|| <= ir_tol ||b|| (cfg.ir_tol, or
 * 1e-9 when 0).  The first iterate of a P-MBF column is the network's
 * prediction for it; of a U-MBF column, -beta s times the prediction of the
 * same basis; of the particular column, zero.  Subdomains with a column
 * that does not reach the tolerance are factored and solved again in FP64
 * (the direct fallback, cfg.fallback_cap slots at a time; counted by
 * mrcm_read_fallback).  Then the traces, as mrcm_solve_mbf.
 *  net, pred  the network and its predictions, FP32 [n_pred][D][H][W] in the
 *             sample order of mrcm_net_samples; pred NULL = every column from zero
 *  f          device FP64 [nz][ny][nx] source density
 * The first call allocates a small column table owned by the handle (make it
 * before any stream capture).  CG iterations: mrcm_read_cg_iterations. */
mrcm_status mrcm_solve_mbf_learned(mrcm_handle* h, const mrcm_net* net, const float* pred, int n_pred,
                                   const double* f, int cg_maxit, int max_outer, void* ws, void* stream);

/* Conjugate-gradient iterations of the last mrcm_solve_mbf_learned, summed over
 * columns (read back synchronously). */
mrcm_status mrcm_read_cg_iterations(mrcm_handle* h, void* ws, long long* iters);

/* FP32 conjugate gradients on the Jacobi-scaled local system of each of the
 * first n_samples samples (order of mrcm_net_samples), from x0[s] (unscaled
 * guess in the sample layout; NULL = zero), to ||r|| <= tol ||b|| or maxit
 * iterations.  The result replaces the P-MBF column in the MBF array (so the
 * FP64 direct solve can check it first); iters[s] (device int) receives the
 * iterations, maxit + 1 when the tolerance was not reached. */
mrcm_status mrcm_pcg_mbf(mrcm_handle* h, const mrcm_net* net, void* ws, const float* x0, int n_samples,
                         int maxit, double tol, int* iters, void* stream);

/* Release the handle and its device tables (not the caller's buffers). */
void mrcm_destroy(mrcm_handle* h);

/* Message of the handle's last failure; with h == NULL, the message of the
 * last failed mrcm_setup on the calling thread. */
const char* mrcm_last_error(const mrcm_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_H */
