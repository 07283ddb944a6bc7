// Internal declarations of the SDD CUDA library (sm_103a).  Not part of the ABI.
//
// Kernels:
//   sdd_prep.cu   monitor on the current mesh + FD gradient + packing (Sec. 3.4), moving-boundary
//                 1-D step, Dirichlet rims and interface scatter (Sec. 3.5), mesh quality (Eq. 8)
//   sdd_mc.cu     interface Monte Carlo (Sec. 3.4): one path per lane, Philox4x32-10,
//                 Euler-Maruyama, exit tests, terminal values, deterministic reductions,
//                 round plan, interface-sampling interpolation
//   sdd_solve.cu  subdomain solves (Sec. 3.5): backward Euler by multigrid-preconditioned CG with
//                 FP64 refinement, or forward-Euler substeps; one CTA (or a cluster of four,
//                 for large subdomains) per subdomain
// Host code:
//   sdd_api.cu    the C ABI of single problems; sdd_batch.cu batches; sdd_server.cu serving;
//                 sdd_noalloc.cu the allocation-free interface Monte Carlo
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

namespace sdd {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// key bumped by the Weyl increments between rounds.
// ---------------------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // high and low words of the 32 x 32 -> 64-bit products (on the device as two 32-bit
        // multiplies, measured faster than one widening multiply)
#ifdef __CUDA_ARCH__
        const uint32_t h0 = __umulhi(kM0, c.x), l0 = kM0 * c.x;
        const uint32_t h1 = __umulhi(kM1, c.z), l1 = kM1 * c.z;
#else
        const uint64_t p0 = (uint64_t)kM0 * c.x, p1 = (uint64_t)kM1 * c.z;
        const uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0;
        const uint32_t h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
#endif
        c = U4{h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
        k0 += kW0;
        k1 += kW1;
    }
    return c;
}

// The same generator with its ten round keys given: rk[2r], rk[2r + 1] is the key of round r
// (key0 + r W0, key1 + r W1).  A launch over one problem reads them from its parameter block,
// so no key arithmetic runs per call.
__device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const uint32_t* rk)
{
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(kM0, c.x), l0 = kM0 * c.x;
        const uint32_t h1 = __umulhi(kM1, c.z), l1 = kM1 * c.z;
        c = U4{h1 ^ c.y ^ rk[2 * r], l1, h0 ^ c.w ^ rk[2 * r + 1], l0};
    }
    return c;
}

// Round keys of philox4x32_10_rk for the 64-bit seed (key0 = low word, key1 = high word).
inline void philox_round_keys(uint64_t seed, uint32_t rk[20])
{
    uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Uniform in (0, 1) from one word without rounding: FP32 keeps the top 23 bits,
// u = (floor(w / 2^9) + 1/2) 2^-23; FP64 u = (w + 1/2) 2^-32.  Built from the exponent bits
// of [1, 2): 1 + k 2^-23 (resp. 1 + w 2^-32) minus (1 - 2^-24) (resp. 1 - 2^-33); the
// difference is representable, so the subtraction is exact.
__device__ __forceinline__ float uniform_open(uint32_t w, float)
{
    // w >> 9 < 2^23, so adding the exponent bits equals or-ing them (one shift-and-add)
    return __int_as_float((w >> 9) + 0x3F800000u) - 0x1.fffffep-1f;
}
__device__ __forceinline__ double uniform_open(uint32_t w, double)
{
    return __hiloint2double((int)(0x3FF00000u | (w >> 12)), (int)(w << 20)) - 0x1.ffffffffp-1;
}

// ---------------------------------------------------------------------------------------
// Packed per-node data read by the path kernel.
// ---------------------------------------------------------------------------------------
template <typename T> struct alignas(4 * sizeof(T)) Mon4 {
    T w, wx, we, pad;  // omega, d omega / d xi, d omega / d eta
};
// Packed monitor of the path kernel.  FP64: one Mon4 per grid node (j nx + i).  FP32: one 64-byte
// cell record per grid node (j nx + i) holding the Mon4 of the corners (i, j), (i + 1, j),
// (i, j + 1), (i + 1, j + 1) of the cell to its upper right, corner indices clamped to the grid
// (the records of the last column and row serve coordinates exactly on the far sides, where the
// clamped corners carry zero weight), so that a bilinear gather is two aligned 32-byte loads of
// one cache line and needs no clamp of the cell index.
inline size_t mon_bytes(int nx, int ny, bool fp64)
{
    return (size_t)nx * ny * (fp64 ? sizeof(Mon4<double>) : 4 * sizeof(Mon4<float>));
}
template <typename T> struct alignas(2 * sizeof(T)) Disp2 {
    T X, Y;            // previous mesh minus the identity: x - Lx xi, y - Ly eta
};

// Per-task partial sums written by one warp (deterministic order).
struct alignas(16) TaskSlot {
    double s1x, s2x, s1y, s2y;   // shifted sums of the path values and their squares
    unsigned long long steps;    // substeps taken
    unsigned long long paths;    // paths completed
};

enum AccMode { kAcc64 = 0, kAccKahan32 = 1 };

// Paths handed to one warp at a time (64 per lane on average): the default task size.  A
// problem's task size may be 1024, 2048 or 4096 (sdd_set_mc_config); a round then gives a node at
// most kTasksPerRound tasks, so the task slots per node stay the same.
constexpr int kPathsPerTask = 2048;
constexpr int kTasksPerRound = 256;
constexpr int kRoundsAhead = 2;  // adaptive Monte Carlo rounds queued ahead of the host's decision
// Adaptive chunk totals are multiples of this many paths.
constexpr int64_t kAdaptiveGranule = 1024;

// Per-problem inputs of the path kernel.
template <typename T> struct McProblem {
    const Mon4<T>* mon;        // packed monitor (mon_bytes: node records, or FP32 cell records)
    const Disp2<T>* disp;      // nx*ny packed displacement of the previous mesh
    const int2* nodes;         // the problem's interface nodes (i, j), by local node id
    int nx, ny, periodic, form, K, bicubic, bb;
    T cb;                      // ds / tau
    T Lx, Ly;
    uint32_t key0, key1, tstep;
    int32_t node_offset;       // global index of the problem's node 0 in the launch's node arrays
    uint32_t rk[20];           // Philox round keys of (key0, key1) (single-problem launches)
    uint32_t cell_bias;        // (nx + 1) * 0x4B000000 mod 2^32: see monitor_at
    float gs[2];               // FP32 Dirichlet cell location: nx - 1, ny - 1 (see monitor_at)
    uint32_t cell_last;        // nx ny - 1: the last FP32 cell record
    const T* bnd;              // moving boundary: tangential boundary coordinates (null: identity)
};

// Grid constants of a problem record for the FP32 cell location (set_grid_consts).
template <typename T>
inline void set_grid_consts(McProblem<T>& R)
{
    R.cell_bias = (uint32_t)(R.nx + 1) * 0x4B000000u;
    R.gs[0] = (float)(R.nx - 1);
    R.gs[1] = (float)(R.ny - 1);
    R.cell_last = (uint32_t)R.nx * (uint32_t)R.ny - 1u;
}

template <typename T> struct McParams {
    McProblem<T> prob;         // single-problem launches
    const McProblem<T>* probs; // batched launches: one record per problem (device memory)
    const int32_t* node_prob;  // batched launches: problem of each global node
    const double* shift;       // global nodes x 2: estimator shifts (node's previous position)
    // round plan (written by the plan kernel), over global node indices
    const int32_t* node_of;    // active node ids
    const int64_t* p_begin;    // first path index of each active node's chunk
    const int64_t* p_count;    // chunk length
    const int64_t* task_off;   // exclusive prefix of tasks per active node (n_active + 1)
    const int32_t* n_active;   // device scalar
    int32_t* task_counter;     // dynamic task dispenser (reset by the plan kernel)
    TaskSlot* slots;           // one per task
    int32_t task_paths;        // paths per task (0: kPathsPerTask)
    // debug records (null unless the debug variant runs; single-problem launches only)
    double* dbg_val;
    int32_t* dbg_steps;
    int8_t* dbg_side;
    int64_t dbg_p0;            // first recorded path index
    int64_t dbg_n;             // recorded paths
};

struct PlanParams {
    int M;
    int64_t* n_done;           // paths accumulated per node
    int64_t* next_total;       // scheduled total per node
    int32_t* node_of;
    int64_t* p_begin;
    int64_t* p_count;
    int64_t* task_off;
    int32_t* n_active;
    int32_t* task_counter;
    int32_t* host_n_active;    // mapped pinned host word
    // optional planning order: M positions taken from n_ranges pool ranges in list order
    const int32_t* range_off;  // first node of each range (null: positions are node ids)
    const int32_t* range_pre;  // exclusive prefix of the range lengths (n_ranges + 1)
    int n_ranges;
    int64_t max_tasks;         // > 0: cap on the round's tasks (nodes in planning order)
    int32_t task_paths;        // paths per task (0: kPathsPerTask); a node takes at most
                               // kTasksPerRound tasks per round
};

struct ReduceParams {
    const int32_t* node_of;
    const int64_t* p_count;
    const int64_t* task_off;
    const int32_t* n_active;
    const TaskSlot* slots;
    const double* shift;
    double* acc;               // M x 4 cumulative shifted sums
    int64_t* n_done;
    int64_t* steps;
    int64_t* paths_run;        // M: paths completed per node (check)
    int64_t* next_total;
    double se_target;          // 0: fixed N
    int64_t max_paths;
};

struct PrepParams {
    int nx, ny, periodic, kind, n_params, precision;
    double Lx, Ly, t;
    const double* t_dev;       // if set, the time is read from device memory (graph replays)
    const double* x;           // current mesh
    const double* y;
    const double* omega_in;    // nodal monitor (kind == NODAL)
    double params[64];
    double* om64;              // out: omega at the nodes (FP64)
    double* wxi64;             // out: FD gradient (FP64)
    double* weta64;
    void* mon;                 // out: Mon4<T>
    void* disp;                // out: Disp2<T>
    int32_t* bad;              // out (nullable): set to 1 if omega <= 0 or anything is not finite
    // moving boundary (Sec. 2): one backward-Euler step of the 1-D generator along each side
    int moving_boundary, form;
    double r;                  // dt / tau
    double* bnd64;             // out: [x on eta=0 (nx), x on eta=1 (nx), y on xi=0 (ny), y on xi=1 (ny)]
    void* bnd;                 // out: the same in the path precision
    double* bnd_scratch;       // 2 (2 nx + 2 ny) doubles
};

// Per-problem record of a batch step's batched launches (monitor and packing, moving boundary,
// estimator shifts, Dirichlet scatter, copy of the new mesh).
struct BatchRec {
    PrepParams prep;           // prep.x, prep.y: the current mesh (written by the copy-back)
    const int2* nodes;         // the problem's interface nodes
    int node_offset;           // global index of its node 0 in the batch's node arrays
    double* xnew;              // the new mesh: rims in, interiors out
    double* ynew;
};

struct SolveParams {
    int nx, ny, px, py, form;
    int scheme;                // 0 backward Euler, 1 forward Euler substeps
    int fe_max_substeps;
    double r;                  // dt / tau
    double rtol;
    int max_iter;
    const double* om64;        // omega at the nodes
    const double* xcur;        // previous mesh (right-hand side)
    const double* ycur;
    double* xnew;              // new mesh: rims in, interiors out
    double* ynew;
    double* ce64;              // east-face coefficients r w_{i+1/2,j} / h_xi^2   (nx*ny)
    double* cn64;              // north-face coefficients r w_{i,j+1/2} / h_eta^2 (nx*ny)
    void* ce;                  // the same in the inner precision
    void* cn;
    void* vec;                 // inner vectors: 4 x nx*ny pairs (e, r, p, q), rims zero
    void* mg;                  // multigrid workspace: mg_stride bytes per subdomain
    size_t mg_stride;
    int32_t* stat_iters;       // per subdomain: PCG iterations, refinement sweeps, converged
    int32_t* stat_outer;
    int32_t* stat_ok;
    double* stat_res;          // per subdomain: final relative residual (max of x, y)
};

// Subdomain lines of an n-node direction split into P parts: part I spans nodes
// split_line(I) .. split_line(I + 1) (equal parts when P divides n - 1).
__host__ __device__ inline int split_line(int I, int n, int P)
{
    return (int)(((int64_t)I * (int64_t)(n - 1)) / (int64_t)P);
}

// Large subdomains are solved by a cluster of kCoopWidth CTAs (sdd_solve.cu): those with at
// least kCoopUnknowns interior unknowns.
constexpr int kCoopWidth = 4;
constexpr int64_t kCoopUnknowns = 32768;

// One CTA's work in a cooperative solve launch: subdomain `sub` of problem `prob`, solved by a
// team of `width` CTAs (kCoopWidth: this CTA's cluster; 1: this CTA alone; 0: idle).
struct SolveItem {
    int32_t prob, sub, width, pad;
};

// Work items of a solve launch over the given subdomains (problem, subdomain, interior unknowns),
// in the given order: a cooperative subdomain takes a whole cluster; the others are packed
// kCoopWidth to a cluster.  Empty when no subdomain is cooperative (the one-CTA kernels serve).
std::vector<SolveItem> solve_items(const std::vector<std::pair<int64_t, int2>>& subs);

// Multigrid hierarchy of an n x m subdomain interior: the coarse grid keeps the nodes of odd
// index, (n - 1) / 2 of them for odd n and n / 2 for even n (then the last coarse node lies one
// fine spacing from the rim); levels while both sizes are >= 3.
__host__ __device__ inline int mg_coarse(int n) { return (n & 1) ? (n - 1) / 2 : n / 2; }
__host__ __device__ inline int mg_levels(int n, int m)
{
    int l = 1;
    while (n >= 3 && m >= 3 && l < 16) {
        n = mg_coarse(n);
        m = mg_coarse(m);
        ++l;
    }
    return l;
}
__host__ __device__ inline size_t mg_align(size_t b) { return (b + 255) / 256 * 256; }
__host__ __device__ inline size_t mg_bytes(int n, int m, size_t real_bytes)
{
    const int L = mg_levels(n, m);
    size_t total = 0;
    for (int l = 0; l < L; ++l) {
        const size_t nn = (size_t)n * m;
        total += 3 * mg_align(nn * 2 * real_bytes) + mg_align((size_t)(n + 1) * m * real_bytes) +
                 mg_align((size_t)n * (m + 1) * real_bytes) + mg_align(nn * real_bytes);
        n = mg_coarse(n);
        m = mg_coarse(m);
    }
    return total;
}

// Interpolated interface node (interface sampling, Sec. 3.6): est[m] = w va + (1 - w) vb with
// v = (node >= 0 ? est[node] : 0) + offset for each of the two anchors a, b.
struct InterpRule {
    int32_t m, a, b, pad;
    double w;
    double oax, oay, obx, oby;
};

// Launchers (return cudaGetLastError of the launch).
cudaError_t launch_prep(const PrepParams& P, cudaStream_t s);
cudaError_t launch_quality(int nx, int ny, const double* x, const double* y, double* q, double* stats,
                           cudaStream_t s);
cudaError_t launch_shift(const int2* nodes, int M, int nx, const double* x, const double* y,
                         double* shift, cudaStream_t s);
// bnd64 (nullable): the moving boundary's new tangential coordinates (PrepParams layout)
cudaError_t launch_scatter(int nx, int ny, int periodic, double Lx, double Ly, const int2* nodes,
                           int M, const double* est, double* xnew, double* ynew, cudaStream_t s,
                           const double* bnd64 = nullptr);
// role (nullable): per node, -1 = estimated by Monte Carlo, >= 0 = interpolated (never planned)
// Nodes outside [lo, hi) (hi < 0: M) and interpolated nodes (role >= 0) are scheduled no paths.
cudaError_t launch_mc_init(int M, int64_t n0, int64_t max_paths, double* acc, int64_t* n_done,
                           int64_t* steps, int64_t* paths_run, int64_t* next_total, cudaStream_t s,
                           const int32_t* role = nullptr, int lo = 0, int hi = -1);
cudaError_t launch_interp(const InterpRule* rules, int n, double* est, double* se, cudaStream_t s);
cudaError_t launch_plan(const PlanParams& P, cudaStream_t s);
template <typename T>
// tpb: threads per block of batched launches (128, 256, 512); batch_mode: the problem switches
// every problem of a batch shares (bit 0 periodic, 1 generator form, 2 bridge test), or -1
cudaError_t launch_mc(const McParams<T>& P, int acc_mode, bool debug, bool batch, int grid, cudaStream_t s,
                      int tpb = 256, int batch_mode = -1);
template <typename T> int mc_max_blocks_per_sm(int acc_mode, bool debug, bool batch, int tpb = 256);
cudaError_t launch_reduce(const ReduceParams& P, int M, cudaStream_t s);
cudaError_t launch_output(int M, const double* acc, const int64_t* n_done, const double* shift,
                          double* est, double* se, cudaStream_t s);
cudaError_t launch_solve(const SolveParams& P, bool fp64_inner, cudaStream_t s);
cudaError_t launch_faces(const SolveParams& P, bool fp64_inner, cudaStream_t s);
// Batched launches of a batch step (blk_off: per-problem block offsets of grid-sized work, n + 1
// entries, blocks of 256 threads as batch_blocks gives them; node work over the concatenated nodes).
int batch_blocks(long n_nodes);
cudaError_t launch_prep_batch(const BatchRec* R, const int32_t* blk_off, int n, int total_blocks, bool fp64,
                              bool any_moving, cudaStream_t s);
cudaError_t launch_shift_batch(const BatchRec* R, const int32_t* node_prob, int M, double* shift, cudaStream_t s);
cudaError_t launch_scatter_batch(const BatchRec* R, const int32_t* blk_off, int n, int total_blocks,
                                 const int32_t* node_prob, int M, const double* est, cudaStream_t s);
cudaError_t launch_copy_back_batch(const BatchRec* R, const int32_t* blk_off, int n, int total_blocks, cudaStream_t s);
cudaError_t launch_faces_batch(const SolveParams* probs, const int32_t* blk_off, int n, int total_blocks,
                               bool fp64_inner, cudaStream_t s);
// order (nullable): (problem, subdomain) of each CTA
cudaError_t launch_solve_batch(const SolveParams* probs, const int32_t* sub_off, int n, int total_subs,
                               bool fp64_inner, cudaStream_t s, bool any_be = true, bool any_fe = false,
                               const int2* order = nullptr);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                          cudaStream_t s);
cudaError_t launch_unit_math(const uint32_t* w, int64_t n, float* out, cudaStream_t s);
// Cooperative solve launches (items from solve_items); the single-problem one also computes the
// face coefficients first, as launch_solve does.
cudaError_t launch_solve_items(const SolveParams& P, const SolveItem* items, int n_items, bool fp64_inner,
                               cudaStream_t s);
cudaError_t launch_solve_batch_items(const SolveParams* probs, const SolveItem* items, int n_items,
                                     bool fp64_inner, cudaStream_t s);

// Host/device shared scheduling rule of the adaptive estimator.
__host__ __device__ inline int64_t adaptive_next_total(int64_t n_done, double se, double target,
                                                       int64_t max_paths)
{
    if (se <= target || n_done >= max_paths) return n_done;
    const double r = se / target;
    const double want = ((double)n_done * (r * r)) * 1.03;
    double total = ceil(want / (double)kAdaptiveGranule) * (double)kAdaptiveGranule;
    const double floor_total = (double)(n_done + kAdaptiveGranule);
    if (total < floor_total) total = floor_total;
    if (total > (double)max_paths) total = (double)max_paths;
    return (int64_t)total;
}

}  // namespace sdd
