/*
 * sdd.h -- C ABI of the GB300 stochastic domain decomposition (SDD) mesh generator.
 *
 * The method (Bihlo, Haynes & Walsh, "Stochastic domain decomposition for time dependent
 * adaptive mesh generation"): the mesh map x(xi, eta, t) of the linearised parabolic mesh
 * generator (Eq. 4; monitor frozen over a step, Sec. 2 and Sec. 3.2) is advanced one time
 * step by
 *   1. Monte Carlo evaluation of its stochastic representation (Eq. 5a Dirichlet, Eq. 6
 *      periodic) at the nodes of the artificial subdomain interfaces, with paths of the SDE
 *      of Eq. (5b) stepped by the Euler-Maruyama scheme of Eq. (7) (Sec. 3.4), then
 *   2. independent deterministic subdomain solves that take those values as Dirichlet data
 *      (Sec. 3.5, Sec. 3.6).
 *
 * Generator forms.  SDD_FORM_DIV is  tau x_t = div(omega grad x)  with the SDE
 * dX = grad(omega)/tau ds + sqrt(2 omega/tau) dW.  SDD_FORM_WINSLOW is the paper's Eq. (4),
 * tau x_t = grad(omega)/omega . grad x + lap x  with dX = grad(omega)/(omega tau) ds +
 * sqrt(2/tau) dW (tau = 1 gives Eq. 4 and Eq. 5b exactly).  Subdomains are stepped by
 * backward Euler with centred 5-point differences and face-averaged coefficients.
 *
 * Conventions for every call.
 *   - Every call returns an sdd_status; no exception crosses the ABI.  sdd_last_error()
 *     returns a thread-local message for the last failing call of the calling thread.
 *   - Grids are row-major, [j * nx + i], i along xi (fast), j along eta (slow).
 *   - Array arguments may be host or device pointers (unified addressing decides);
 *     the library copies inputs and never keeps a caller's pointer.  Outputs are
 *     caller-owned.  When an output is host memory the call returns after it is written;
 *     device outputs are written in order on the problem's stream.
 *   - All device work runs on the stream given to sdd_create_problem / sdd_set_stream.
 *   - A problem object owns its device memory and must be used from one host thread
 *     at a time.
 *   - Failures of the CUDA runtime return SDD_ERR_CUDA; the problem is then unusable
 *     and should be destroyed.
 */
#ifndef SDD_H
#define SDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdd_problem sdd_problem;

typedef enum {
    SDD_OK = 0,
    SDD_ERR_INVALID_ARG = 1,     /* a size, a flag or a pointer is out of its documented range */
    SDD_ERR_OOM = 2,             /* device or pinned-host allocation failed                    */
    SDD_ERR_CUDA = 3,            /* a CUDA runtime call failed (message in sdd_last_error)     */
    SDD_ERR_NOT_CONVERGED = 4,   /* a subdomain solve hit solve_max_iter; the best iterate is kept */
    SDD_ERR_SE_NOT_REACHED = 5,  /* adaptive MC hit max_paths_per_node before se_target at some node */
    SDD_ERR_NO_DEVICE = 6,       /* no CUDA device is visible                                  */
    SDD_ERR_CANCELLED = 7        /* a served request was cancelled before it was finished       */
} sdd_status;

enum { SDD_FORM_DIV = 0, SDD_FORM_WINSLOW = 1 };

/* Working precision of the paths and of the estimator sums (subdomain solves: FP64 PCG for
 * SDD_FP64, FP32 PCG with FP64 residuals and iterative refinement otherwise). */
enum { SDD_FP64 = 0, SDD_FP32_ACC64 = 1, SDD_FP32_KAHAN = 2 };

/* Monitor (mesh density) kinds, evaluated on the current physical mesh (x, y) at t^n. */
enum {
    SDD_MONITOR_NODAL = 0, /* values supplied with sdd_set_monitor                              */
    SDD_MONITOR_GAUSS = 1, /* sqrt(1 + a exp(-b |x - c|^2)); params a, b, cx, cy                */
    SDD_MONITOR_FRONT = 2, /* sqrt(1 + alpha |grad u|^2), u = tanh(R (|x - c| - r0 - v t));
                              params alpha, R, r0, v, cx, cy (the arc-length monitor, Sec. 1)   */
    SDD_MONITOR_BUMPS = 3, /* 1 + sum_k a_k exp(-|x - c_k|^2 / w_k^2); params (a, w, cx, cy)*   */
    SDD_MONITOR_RINGS = 4  /* sqrt(1 + alpha |grad u|^2), u = sum_k tanh(R (|x - c_k|^2 - r2));
                              params alpha, R, r2, (cx, cy)* (the five-ring problem, Sec. 4.2)  */
};

typedef struct {
    int32_t nx, ny;          /* grid nodes per direction, >= 3, nx * ny <= 2^28                      */
    int32_t px, py;          /* subdomains per direction, 1 <= px <= nx - 1, 1 <= py <= ny - 1;
                                subdomain I spans node columns floor(I (nx-1)/px) ..
                                floor((I+1)(nx-1)/px) (equal when px divides nx - 1), likewise J;
                                the interface nodes they give must number below 2^23          */
    int32_t periodic;        /* 0: Dirichlet, boundary mesh fixed at (Lx xi, Ly eta) (Sec. 2);
                                1: doubly periodic, x(xi+1) = x(xi) + Lx, y(eta+1) = y(eta) + Ly    */
    int32_t form;            /* SDD_FORM_DIV or SDD_FORM_WINSLOW                                   */
    int32_t precision;       /* SDD_FP64, SDD_FP32_ACC64 or SDD_FP32_KAHAN                          */
    int32_t bicubic;         /* 1: Keys bicubic of the previous mesh at the path end (Sec. 3.4);
                                0: bilinear                                                          */
    int32_t bb_test;         /* 1: Brownian-bridge crossing test between substeps (Sec. 3.4)       */
    int32_t substeps;        /* K in [1, 2^20]: Euler-Maruyama substeps per step, ds = dt / K (Eq. 7) */
    int32_t solve_max_iter;  /* PCG iteration cap per subdomain solve, >= 1                       */
    int32_t iface_stride;    /* 0 or 1: Monte Carlo at every interface node; k in [2, 2^16]: at
                                every k-th node of each interface line (index along the line a
                                multiple of k) and at line crossings, the other nodes linearly
                                interpolated along their line between the nearest sampled nodes
                                or the line's end (Sec. 3.6: "a sample can be evaluated with the
                                rest obtained by interpolation").  Sampled nodes keep their node
                                ids, so their estimates equal those of k = 1.                  */
    double Lx, Ly;           /* physical rectangle [0, Lx] x [0, Ly], > 0                           */
    double tau;              /* relaxation time of the generator, > 0                              */
    double dt;               /* mesh time step, > 0                                                */
    uint64_t seed;           /* Philox key                                                         */
    int64_t paths_per_node;  /* N >= 2: paths per node (fixed mode) or first chunk (adaptive)     */
    int64_t max_paths_per_node; /* adaptive cap, >= paths_per_node, <= 2^31                       */
    double se_target;        /* > 0: adaptive -- draw paths until max(SE_x, SE_y) <= se_target
                                at every node; 0: fixed N                                           */
    double solve_rtol;       /* subdomain solves stop at ||b - A x||_2 <= solve_rtol ||b||_2, > 0   */
    double t0;               /* time of the initial mesh                                           */
    int32_t subdomain_scheme; /* 0: backward Euler (default, any step size); 1: forward Euler, the
                                paper's local solver (Sec. 3.5), in S = ceil(max_P sum_nb c_nb/d_P)
                                explicit substeps (every substep a convex combination: discrete
                                maximum principle) with the rim values interpolated linearly in
                                time between the previous mesh and the new Dirichlet data      */
    int32_t fe_max_substeps; /* forward Euler: a subdomain needing more substeps is not solved
                                (SDD_ERR_NOT_CONVERGED, interior left at x^n); 0 means 2^16     */
    int32_t moving_boundary; /* 0: boundary mesh fixed at (Lx xi, Ly eta); 1 (Dirichlet only): the
                                tangential components -- x along eta = 0, 1 and y along xi = 0, 1 --
                                take one backward-Euler step of the 1-D generator along their side
                                before the interface Monte Carlo (Sec. 2); exiting paths then take
                                the new boundary mesh, linearly interpolated along the exit side.
                                The normal components and the corners stay fixed.            */
} sdd_params;

typedef struct {
    int32_t M;                  /* interface nodes                                             */
    int32_t step_index;         /* n: steps taken so far (fourth Philox counter word)          */
    double t;                   /* current time t^n = t0 + n dt                                */
    int64_t path_steps;         /* substeps actually taken by all paths of the last MC call    */
    int64_t paths;              /* paths run by the last MC call                               */
    int32_t mc_rounds;          /* launches of the last MC call (1 in fixed mode)              */
    int32_t nodes_not_reached;  /* nodes above se_target after the last adaptive MC call       */
    double max_se;              /* largest SE over nodes and components (last MC call)         */
    int32_t solve_iters_max;    /* largest total PCG iteration count over subdomains (last solve) */
    int32_t solve_outer_max;    /* largest refinement sweep count over subdomains (last solve)  */
    double solve_rel_residual;  /* largest final ||b - A x|| / ||b|| over subdomains and components */
    double mc_kernel_ms;        /* device time of the path-kernel launches of the last MC call,
                                   CUDA events on the problem's stream                          */
    int32_t mc_kernel_launches; /* path-kernel launches of the last MC call                     */
    int32_t reserved1;
    int64_t kernel_launches;    /* kernels launched by this problem since creation              */
    double solve_kernel_ms;     /* device time of the last subdomain-solve launch(es) (face
                                   coefficients and solves; CUDA events on the stream)          */
} sdd_stats;

/* Create a problem: validates params, copies the initial mesh x0, y0 (nx*ny each, host or
 * device), allocates all device state.  Dirichlet problems require the boundary nodes of
 * x0, y0 to equal (Lx xi, Ly eta) to within 1e-12 (Lx + Ly).  `stream` is a cudaStream_t
 * (NULL = legacy default stream).  Monitor defaults to SDD_MONITOR_NODAL with omega = 1.
 * Sec. 2 (computational square, physical rectangle, fixed boundary), Sec. 3.4 (dt, K, N). */
sdd_status sdd_create_problem(const sdd_params* params, const double* x0, const double* y0,
                              void* stream, sdd_problem** out);

/* Release every resource of the problem (NULL is ignored). */
void sdd_destroy_problem(sdd_problem* p);

/* Replace the stream all later work of the problem is ordered on. */
sdd_status sdd_set_stream(sdd_problem* p, void* stream);

/* Overwrite the current mesh x^n, y^n (nx*ny each).  Same boundary rule as at creation. */
sdd_status sdd_set_mesh(sdd_problem* p, const double* x, const double* y);

/* Copy the current mesh x^n, y^n out (nx*ny each). */
sdd_status sdd_get_mesh(sdd_problem* p, double* x, double* y);

/* Nodal monitor omega (nx*ny values, > 0), frozen until replaced (Sec. 3.2).  Periodic
 * problems read only the nodes i < nx-1, j < ny-1 (the wrap nodes repeat node 0). */
sdd_status sdd_set_monitor(sdd_problem* p, const double* omega);

/* Analytic monitor re-evaluated on the current mesh at t^n before each MC call and step
 * (the MP procedure: omega from u^n on x^n, Sec. 2 and Sec. 3.6).  Periodic problems use
 * the minimum-image offset x - c.  n_params: 4 (GAUSS), 6 (FRONT), 4k with k <= 16 (BUMPS),
 * 3 + 2k with 1 <= k <= 30 (RINGS). */
sdd_status sdd_set_monitor_analytic(sdd_problem* p, int32_t kind, const double* params,
                                    int32_t n_params);

/* Interface Monte Carlo (Sec. 3.4): for every interface node m, paths p = 0, 1, ... of
 * Eq. (7) started at the node, each substep k drawing Philox4x32-10 with counter
 * (k, p, m, n) and key = seed, estimate x^{n+1} and y^{n+1} by the arithmetic mean.
 * Outputs (nullable): est_xy, se_xy: M x 2 doubles (node-major, x then y);
 * paths_used: M int64.  Does not advance time.  Returns SDD_ERR_SE_NOT_REACHED (outputs
 * still written) when an adaptive node hit max_paths_per_node, and SDD_ERR_INVALID_ARG (no
 * outputs) when the monitor is not finite and > 0 at every node or the mesh is not finite
 * (checked on the device during the call). */
sdd_status sdd_interface_mc(sdd_problem* p, double* est_xy, double* se_xy, int64_t* paths_used);

/* Subdomain solves (Sec. 3.5): Dirichlet data = iface_xy (M x 2, nullable = the last
 * sdd_interface_mc result) on the interfaces and the boundary mesh on the physical boundary;
 * backward-Euler 5-point solve of every subdomain interior.  Writes the new mesh to x_out,
 * y_out (nx*ny each, nullable).  Does not advance time. */
sdd_status sdd_subdomain_solve(sdd_problem* p, const double* iface_xy, double* x_out, double* y_out);

/* A time step split by interface nodes (for a problem shared by several GPUs): the estimates of
 * Eq. (5a) at different interface nodes are independent given the frozen monitor and mesh
 * (Sec. 3.4: each node's paths use the counter (k, p, m, n) of their own node id m), so each
 * part of [0, M) can be computed apart and the parts assembled.
 *
 * sdd_interface_mc_range: sdd_interface_mc for the nodes node_begin .. node_end - 1 only
 * (0 <= node_begin <= node_end <= M): the same paths, estimates and standard errors those nodes
 * get in sdd_interface_mc, bit for bit.  est_xy, se_xy (M x 2 doubles) and paths_used (M int64)
 * are full-size arrays (nullable; host or device) of which only the range's entries are
 * written.  SDD_ERR_INVALID_ARG for a range outside [0, M] or a problem with interface sampling
 * (iface_stride > 1: interpolated nodes need every range's estimates); SDD_ERR_SE_NOT_REACHED as
 * sdd_interface_mc, for the range's nodes.  Does not advance time.
 *
 * sdd_step_from_interface: the rest of the step sdd_step takes after its interface Monte Carlo:
 * the subdomain solves (Sec. 3.5) with iface_xy (M x 2 doubles, host or device, required when
 * M > 0) as the interface data, then time and the step index advance and the new mesh is
 * written to x_out, y_out (nullable).  Given the estimates of every node (e.g. the ranges of
 * sdd_interface_mc_range assembled), the new mesh is bitwise that of sdd_step. */
sdd_status sdd_interface_mc_range(sdd_problem* p, int32_t node_begin, int32_t node_end, double* est_xy,
                                  double* se_xy, int64_t* paths_used);
sdd_status sdd_step_from_interface(sdd_problem* p, const double* iface_xy, double* x_out, double* y_out);

/* One alternating step t^n -> t^{n+1} (Sec. 3.6): monitor on x^n at t^n (analytic kinds),
 * interface MC, subdomain solves, then x^n <- x^{n+1}, n <- n + 1.  x_out, y_out nullable.
 * On an invalid monitor or mesh (as sdd_interface_mc) returns SDD_ERR_INVALID_ARG and takes no
 * step. */
sdd_status sdd_step(sdd_problem* p, double* x_out, double* y_out);

/* M^kP step (Sec. 5): t^n -> t^{n+1} as K mesh sub-steps of dt/K.  Before each sub-step the
 * monitor is evaluated on the current sub-mesh at the time t^n of the step (analytic kinds; the
 * paper interpolates rho^n onto the sub-mesh, the analytic monitor is evaluated there exactly;
 * nodal values stay with their nodes), then interface MC and subdomain solves with dt/K.
 * Sub-step k of step n uses n K + k as the fourth Philox counter word, so K = 1 is sdd_step.
 * K in [1, 2^16] with (n + 1) K <= 2^32.  Counters (sdd_get_stats) sum over the sub-steps.  On
 * an error other than SDD_ERR_SE_NOT_REACHED / SDD_ERR_NOT_CONVERGED the problem keeps the last
 * completed sub-mesh and the step index n. */
sdd_status sdd_step_mkp(sdd_problem* p, int32_t K, double* x_out, double* y_out);

/* Counters of the last calls (see sdd_stats). */
sdd_status sdd_get_stats(const sdd_problem* p, sdd_stats* out);

/* ---- Launch configuration of the path kernel (Sec. 3.4's N paths per node) -----------------
 * The path kernel is a persistent grid of blocks_per_sm x SMs blocks of threads_per_block
 * threads; each warp takes tasks of paths_per_task consecutive paths of one node, and a
 * Monte Carlo round gives a node at most 256 tasks (256 x paths_per_task paths).
 *   threads_per_block : 128, 256 or 512 for batches (sdd_batch_set_mc_config); 256 for a
 *                       single problem.
 *   blocks_per_sm     : 1 .. max_blocks_per_sm, the register limit of the kernel (read-only
 *                       field, filled by the get calls; ignored by the set calls).
 *   paths_per_task    : 1024, 2048 (the default) or 4096.
 * What does and does not change results: threads_per_block and blocks_per_sm never do (every
 * warp runs whole tasks of fixed paths, and the sums are reduced task by task in a fixed order).
 * paths_per_task groups a node's paths differently for the estimator sums (per lane, per task,
 * per round): FP64 estimates then differ in the last bits (about 1e-16 relative per sum), and in
 * the adaptive mode a node whose SE lies within that of the target may take another chunk.  A
 * batch uses one paths_per_task for all its problems, so a batched problem gives bitwise the
 * results of stepping it alone with the same paths_per_task.  The configuration is not part of
 * a checkpoint (sdd_save). */
typedef struct {
    int32_t threads_per_block;
    int32_t blocks_per_sm;
    int32_t paths_per_task;
    int32_t max_blocks_per_sm;
} sdd_mc_config;

/* The problem's current configuration. */
sdd_status sdd_get_mc_config(const sdd_problem* p, sdd_mc_config* out);

/* Set the configuration (0 in a field keeps its current value; blocks_per_sm 0 = the maximum).
 * SDD_ERR_INVALID_ARG for values outside the lists above. */
sdd_status sdd_set_mc_config(sdd_problem* p, const sdd_mc_config* cfg);

/* Autotuner: prepares the next step's first Monte Carlo round (monitor, initial chunk, plan),
 * times one path-kernel launch of that round (the faster of two) at every blocks_per_sm from 1
 * to the maximum and, with tune_paths_per_task = 1, at paths_per_task 1024, 2048 and 4096
 * (otherwise at the current one), keeps the configuration with the least time per path, and
 * writes it to *chosen (nullable).  The launches write only scratch task slots: no state of the
 * problem changes (the next step prepares, initialises and plans again).  Waits for the
 * problem's stream. */
sdd_status sdd_tune(sdd_problem* p, int32_t tune_paths_per_task, sdd_mc_config* chosen);

/* Interface nodes of the problem: ij (M x 2 int32 (i, j), nullable) and *M. */
sdd_status sdd_get_interface_nodes(const sdd_problem* p, int32_t* ij, int32_t* M);

/* Host-only (no GPU needed): interface nodes of an nx x ny grid split px x py, in the
 * order that defines the node id m: vertical interface lines by increasing i (nodes by
 * increasing j), then horizontal lines by increasing j (nodes by increasing i, skipping
 * nodes already listed).  Dirichlet lines: i = I (nx-1)/px, I = 1..px-1, j = 1..ny-2;
 * periodic lines: I = 0..px-1, j = 0..ny-2.  ij may be NULL to query *M.  Sec. 3.1, 3.5. */
sdd_status sdd_interface_layout(int32_t nx, int32_t ny, int32_t px, int32_t py, int32_t periodic,
                                int32_t* ij, int32_t* M);

/* Host-only (no GPU needed): which interface nodes params->iface_stride leaves to Monte Carlo:
 * sampled (M int32, node-id order, nullable) receives 1 for a sampled node and 0 for an
 * interpolated one; *M the node count.  Validates params as sdd_create_problem does. */
sdd_status sdd_interface_sampling(const sdd_params* params, int32_t* sampled, int32_t* M);

/* Host-only: adaptive path total of a node after n_done paths with standard error se
 * (max of both components): n_done when se <= target or n_done >= max_paths, else
 * min(max_paths, max(n_done + 1024, 1024 ceil(1.03 n_done (se/target)^2 / 1024))). */
int64_t sdd_adaptive_next_total(int64_t n_done, double se, double target, int64_t max_paths);

/* Geometric mesh quality of the current mesh (Eq. 8): per cell Q = tr(J^T J) / (2 |det J|),
 * J from the mean of the cell's two xi-edges and two eta-edges, Q >= 1 with equality for a
 * square cell (Sec. 3.7).  q_cells: (nx-1)*(ny-1) doubles, row-major (nullable); *q_max and
 * *q_mean (nullable): the maximum and mean over the cells.  Returns when written. */
sdd_status sdd_mesh_quality(sdd_problem* p, double* q_cells, double* q_max, double* q_mean);

/* Checkpoint of a problem (no counterpart in the paper; the method has no hidden state beyond
 * what is saved, because the Philox counter is the time-step index): parameters, time-step
 * index, monitor (kind, parameters, nodal values) and the current mesh, written to the file
 * `path` in this layout (little-endian): 8 bytes "SDDCKPT1", int32 sizeof(sdd_params), the
 * sdd_params record, int64 step index, int32 monitor kind, int32 parameter count, 64 doubles
 * of monitor parameters, then nx*ny doubles each of x, y and the nodal monitor.  Returns
 * SDD_ERR_INVALID_ARG if the file cannot be written. */
sdd_status sdd_save(sdd_problem* p, const char* path);

/* Resume a problem from a checkpoint written by sdd_save, with its work on `stream`: stepping
 * it continues bit for bit as the saved problem would have.  Returns SDD_ERR_INVALID_ARG for a
 * missing, truncated or foreign file (checked before any device work). */
sdd_status sdd_load(const char* path, void* stream, sdd_problem** out);

/* Test hook: the monitor as frozen for the next MC call (nx*ny each, FP64, nullable):
 * omega and its finite-difference gradient (Sec. 3.4). */
sdd_status sdd_get_monitor(sdd_problem* p, double* omega, double* w_xi, double* w_eta);

/* Test hook: per-path records of paths p_begin .. p_begin + n_paths - 1 of interface node
 * `node`, computed by the same kernel code as sdd_interface_mc: val_xy (n x 2 doubles),
 * exit_step (substeps taken), exit_side (0: xi=0, 1: xi=1, 2: eta=0, 3: eta=1, 4: none).
 * Any output may be NULL.  Uses the current monitor and mesh; does not change state. */
sdd_status sdd_debug_paths(sdd_problem* p, int32_t node, int64_t p_begin, int64_t n_paths,
                           double* val_xy, int32_t* exit_step, int8_t* exit_side);

/* Test hook: n Philox4x32-10 draws on the device (ctr n x 4, key n x 2, out n x 4 words),
 * on the legacy default stream; returns after `out` is written. */
sdd_status sdd_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out);

/* Test hook: the FP32 Box-Muller pieces the path kernel evaluates (Sec. 3.4, the N(0,1) draws of
 * Eq. 7), on n given Philox words w (host or device, n words): out (n x 5 floats) holds, per
 * word, the uniform u = (floor(w / 2^9) + 1/2) 2^-23, the kernel's ln u, its sqrt(-2 ln u) and
 * sin 2 pi u, cos 2 pi u.  On the legacy default stream; returns after `out` is written. */
sdd_status sdd_debug_unit_math(const uint32_t* w, int64_t n, float* out);

/* Test hook: the number of out-of-range gather indices the path kernel met since the library
 * was loaded, in a build compiled with -DSDD_BOUNDS_CHECK.  Such a build checks every monitor,
 * mesh, boundary and queue index before its load; an index outside its array is counted and
 * replaced by 0, so the load stays in bounds.  Returns -1 in a normal build and -2 on a CUDA
 * error.  Waits for the device. */
int64_t sdd_debug_bounds_violations(void);

/* ---- Batches of independent problems ------------------------------------------------------
 * Many problems of uneven grid and subdomain counts advance one alternating step together
 * (Sec. 3.6 for each): per problem the monitor preparation and the scatter of Dirichlet data;
 * ONE persistent path-kernel launch per round for the interface nodes of all problems, and
 * ONE launch for all subdomain solves (one CTA per (problem, subdomain)).  Each problem's
 * results are bitwise those of sdd_step on it alone (own seed, local node ids in the Philox
 * counter, per-node path schedule, fixed-order reductions).  All problems must share
 * precision, se_target and paths_per_node (and max_paths_per_node when adaptive), and their
 * interface nodes must number below 2^23 in total (else SDD_ERR_INVALID_ARG); the batch
 * keeps pointers to them (they must outlive it) and orders its work on `stream`.
 * use_graph = 1 (fixed N only, stream not NULL): the first step records its launches in a CUDA
 * graph that later steps replay (re-recorded if a problem's mesh buffers change). */
typedef struct sdd_batch sdd_batch;

sdd_status sdd_batch_create(sdd_problem* const* problems, int32_t n, void* stream, int32_t use_graph,
                            sdd_batch** out);

/* One alternating step of every problem of the batch (x^n <- x^{n+1}, n <- n + 1 for each).
 * Returns after queueing the work on the batch's stream. */
sdd_status sdd_batch_step(sdd_batch* b);

/* Threads per block of the batch's path-kernel launches: threads_per_block = 128, 256 (the
 * default) or 512 selects one; 0 tunes it.  Tuning prepares and plans the first Monte Carlo round
 * of the next step, times one path-kernel launch at each size on that plan (each at all the
 * blocks per SM its registers allow) into the scratch task slots, and keeps the fastest.  No
 * problem's state changes, and results never depend on the size: every warp runs whole tasks of
 * fixed paths, reduced in a fixed order.  *chosen (nullable) receives the size in use.  Waits
 * for the batch's and the problems' streams; a recorded CUDA graph is recorded again at the next
 * step.  SDD_ERR_INVALID_ARG for any other size. */
sdd_status sdd_batch_tune(sdd_batch* b, int32_t threads_per_block, int32_t* chosen);

/* Counters of the last batch step over all problems: M, path_steps, paths, mc_rounds,
 * nodes_not_reached, max_se, solve maxima, kernel_launches (since creation), and in
 * mc_kernel_ms the device time of the whole last step and in solve_kernel_ms that of its
 * batched solve launch (CUDA events on the batch's stream).
 * Waits for the batch's stream.  Returns SDD_ERR_INVALID_ARG (counters still written) when a
 * problem's monitor was not finite and > 0 at every node or its mesh not finite in that step. */
sdd_status sdd_batch_get_stats(sdd_batch* b, sdd_stats* out);

/* Launch configuration of the batch's path kernel (sdd_mc_config).  Setting paths_per_task
 * sets it on every problem of the batch as well; a recorded CUDA graph is recorded again at the
 * next step. */
sdd_status sdd_batch_get_mc_config(sdd_batch* b, sdd_mc_config* out);
sdd_status sdd_batch_set_mc_config(sdd_batch* b, const sdd_mc_config* cfg);

/* Autotuner of a batch: as sdd_tune, over threads_per_block 128, 256 and 512, every
 * blocks_per_sm their register limits allow and, with tune_paths_per_task = 1, paths_per_task
 * 1024, 2048 and 4096; the chosen paths_per_task goes to every problem.  Waits for the batch's
 * and the problems' streams.  (sdd_batch_tune tunes threads_per_block alone.) */
sdd_status sdd_batch_tune_mc(sdd_batch* b, int32_t tune_paths_per_task, sdd_mc_config* chosen);

/* Release the batch (not its problems). */
void sdd_batch_destroy(sdd_batch* b);

/* ---- Serving: continuous batching of one-step requests ------------------------------------
 * A server advances independent requests -- one alternating step each (Sec. 3.6) of a mesh
 * problem -- that arrive over time.  Requests join and leave the running set between rounds of
 * the path kernel: a round is ONE persistent path-kernel launch over the interface nodes of all
 * running requests (a shared node pool in which each request holds a contiguous range), and a
 * request whose nodes have all reached the service level is finished at once (estimates,
 * Dirichlet scatter, subdomain solves, on a second stream) while the others keep sampling.
 * A request's result is bitwise that of sdd_step on a problem created alone with the same
 * parameters, mesh, monitor and step index (own seed, local node ids in the Philox counter,
 * per-node path schedule, fixed-order reductions).
 * Admission is first come, first served, bounded by the node pool, the number of resident
 * requests and a device-memory budget; with round_paths set, each round's paths also go to
 * the oldest running requests first, so requests complete close to arrival order instead of
 * all together.  The device state of collected requests is kept per
 * grid shape (nx, ny, px, py, periodic, iface_stride, subdomain_scheme) and reused, so steady-state serving allocates no
 * device memory; cached state is freed (oldest first) only when a new shape needs room.
 * The paper has no serving layer: this is the system around its method. */
typedef struct sdd_server sdd_server;

typedef struct {
    int32_t precision;           /* SDD_FP64 / SDD_FP32_ACC64 / SDD_FP32_KAHAN for every request */
    int32_t max_resident;        /* requests holding device state at once (running, finishing,
                                    or finished but not collected), in [1, 2^16]                */
    int64_t max_nodes;           /* node-pool capacity (interface nodes of resident requests),
                                    in [1, 2^23); each pool node costs about 12.5 KB            */
    int64_t mem_budget_bytes;    /* device bytes for per-request state (pool excluded), 0 = no
                                    limit                                                       */
    double se_target;            /* service level, meaning as in sdd_params (0: fixed N)        */
    int64_t paths_per_node;      /* fixed N, or the first chunk when adaptive, >= 2              */
    int64_t max_paths_per_node;  /* adaptive cap in [paths_per_node, 2^31]                       */
    int64_t round_paths;         /* > 0: paths per round at most, given to running requests
                                    oldest first (a node's chunk is never split, and the first
                                    pending node always runs); 0: every pending chunk each round */
} sdd_server_params;

typedef struct {
    int64_t submitted, completed, collected; /* requests                                        */
    int32_t queued, running, finishing, done; /* requests in each state now                     */
    int64_t rounds;              /* path-kernel rounds launched                                 */
    int64_t kernel_launches;     /* kernels launched by the server                               */
    double mc_kernel_ms;         /* device time of all completed path-kernel rounds (CUDA events) */
    int64_t path_steps;          /* substeps taken by the paths of completed requests            */
    int64_t interface_nodes;     /* interface nodes of completed requests                         */
    int64_t resident_bytes;      /* device bytes of request state held now (cache included)     */
    int64_t cached_bytes;        /* of which kept for reuse                                      */
    int64_t pool_bytes;          /* device bytes of the node pool                                */
    int64_t pool_high_water;     /* highest pool node index + 1 used so far                       */
    int64_t allocations;         /* per-request device-state allocations since creation          */
} sdd_server_stats;

/* Create a server whose work is ordered on `stream` (cudaStream_t, not NULL; a non-blocking
 * stream is best) plus two internal streams (uploads; finishing requests). */
sdd_status sdd_server_create(const sdd_server_params* params, void* stream, sdd_server** out);

/* Queue one request: an alternating step of the problem `params` (precision, se_target,
 * paths_per_node and max_paths_per_node must equal the server's) from the mesh (x0, y0) (HOST
 * memory, nx*ny each, copied) at time-step index step_index >= 0 (fourth Philox counter word;
 * time t0 + step_index dt).  Monitor: an analytic kind with its parameters as for
 * sdd_set_monitor_analytic, or SDD_MONITOR_NODAL with omega (HOST, nx*ny, copied; NULL means
 * omega = 1).  *id receives the request id (increasing from 1).  Does not touch the GPU. */
sdd_status sdd_server_submit(sdd_server* s, const sdd_params* params, const double* x0, const double* y0,
                             int32_t monitor_kind, const double* monitor_params, int32_t n_params,
                             const double* omega, int32_t step_index, int64_t* id);

/* One scheduling round: collect finishing requests whose work is complete, admit queued ones
 * (upload, monitor, node-pool init), plan the next path-kernel round over all running requests,
 * start finishing every request whose nodes are all done, and launch the round.  Waits for the
 * previous round's reductions (one host round trip per round).  Outputs (nullable): requests
 * running and queued after the call.  A request that can never fit the memory budget completes
 * with SDD_ERR_OOM. */
sdd_status sdd_server_progress(sdd_server* s, int32_t* n_running, int32_t* n_queued);

/* Ids of requests completed since the last poll, oldest first (at most cap; the rest wait for
 * the next poll); *n receives the count. */
sdd_status sdd_server_poll(sdd_server* s, int64_t* ids, int32_t cap, int32_t* n);

/* Result of a completed request: the new mesh (x, y: nx*ny each), its interface estimates and
 * standard errors (est_xy, se_xy: M x 2, node-id order), and its counters (st: M, step_index +
 * 1, t, path_steps, paths, mc_rounds = rounds launched while it had pending nodes,
 * nodes_not_reached, max_se, solve maxima).  Host or device pointers, each nullable; returns when host outputs are written.
 * Releases the request (its id becomes invalid).  Returns the request's own status:
 * SDD_ERR_SE_NOT_REACHED or SDD_ERR_NOT_CONVERGED with outputs written; without outputs,
 * SDD_ERR_INVALID_ARG when its monitor was not finite and > 0 at every node or its mesh not
 * finite (found after its first round; no subdomain solve is run), and SDD_ERR_OOM. */
sdd_status sdd_server_result(sdd_server* s, int64_t id, double* x, double* y, double* est_xy, double* se_xy,
                             sdd_stats* st);

/* Cancel a request.  A queued request completes at once; a running one leaves the round plan
 * at the next sdd_server_progress (a round already launched may still sample its nodes) and
 * completes without a subdomain solve; either way sdd_server_result then returns
 * SDD_ERR_CANCELLED without outputs.  A request whose finishing work has started completes
 * normally (the call returns SDD_OK and does nothing).  Unknown or collected ids:
 * SDD_ERR_INVALID_ARG. */
sdd_status sdd_server_cancel(sdd_server* s, int64_t id);

/* Counters of the server (waits for nothing). */
sdd_status sdd_server_get_stats(sdd_server* s, sdd_server_stats* out);

/* Wait for the server's streams and release everything, including uncollected requests. */
void sdd_server_destroy(sdd_server* s);

/* Allocation-free interface Monte Carlo.  The paper has no counterpart: this entry point
 * serves callers that cannot call cudaMalloc -- for instance a host framework whose caching
 * allocator owns the device memory budget and forbids allocations outside it, or a
 * latency-critical loop that cannot afford a device allocation.  It runs the same kernels as
 * sdd_interface_mc in fixed-N mode (same Philox streams, same node ids, same estimates) for
 * the nodal monitor `omega` on the mesh (x, y) at time-step index `step_index`, and allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *   params : as for sdd_create_problem, with se_target == 0 (fixed paths_per_node), every
 *            interface node sampled (iface_stride <= 1), a fixed boundary (moving_boundary ==
 *            0) and an equal split ((nx-1) % px == 0, (ny-1) % py == 0).
 *   x, y, omega : nx*ny doubles in DEVICE memory (read); est_xy, se_xy : M x 2 doubles in
 *            DEVICE memory (written, same layout as sdd_interface_mc).
 *   stream : cudaStream_t for all work (NULL = legacy default stream); the call returns
 *            without waiting for the GPU.
 * Intermediates live in one 16 MiB device array inside the library, held by every GPU that
 * loads it until the process exits.  Requests needing more are rejected with
 * SDD_ERR_INVALID_ARG: the requirement is 96 B per grid node (FP32; 72 B in FP64), 116 B per
 * interface node and 48 B per task of 2048 paths, min(N, 2^19)/2048 tasks per interface node
 * (rounded up), each block aligned to 256 B -- e.g. a 257x257 grid with 1521 interface nodes
 * fits in FP32 for N <= 2.8e5.  Host pointers are rejected.  A problem without interface nodes
 * (one Dirichlet subdomain) returns SDD_OK and writes nothing (est_xy and se_xy may be NULL).
 * The inputs are not validated on the device: the estimates are undefined unless omega is
 * finite and > 0, x and y are finite, and on Dirichlet grids the boundary nodes of (x, y) are
 * the identity mesh (sdd_interface_mc reports such inputs as SDD_ERR_INVALID_ARG instead).
 * The first call with a device current resolves the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.  The address is
 * resolved again when the device's context has changed since (after cudaDeviceReset).
 * Every call shares the array and leaves its contents behind; each call re-initialises what it
 * reads, and calls that overlap on the GPU race.  Errors are reported by the status only
 * (sdd_last_error is not updated by this call). */
sdd_status sdd_interface_mc_noalloc(const sdd_params* params, const double* x, const double* y,
                                    const double* omega, int32_t step_index, double* est_xy,
                                    double* se_xy, void* stream);

const char* sdd_status_string(sdd_status s);
const char* sdd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SDD_H */
