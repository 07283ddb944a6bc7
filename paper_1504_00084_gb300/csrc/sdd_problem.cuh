// Host-side state of one SDD problem (internal; shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sdd.h"
#include "sdd_internal.cuh"

// NVTX range over a host scope (monitor preparation, Monte Carlo rounds, solves, batch steps,
// server progress), for timeline tools; header-only NVTX costs nothing with no tool attached.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

struct sdd_problem {
    sdd_params prm{};
    cudaStream_t stream = nullptr;
    int M = 0;
    std::vector<int32_t> ij;
    int mc_grid = 1;                // persistent path-kernel grid: SMs x mc_blocks_per_sm
    int mc_blocks_per_sm = 1;       // resident path-kernel blocks per SM (sdd_set_mc_config)
    int mc_max_blocks_per_sm = 1;   // the register limit of the path kernel
    int task_paths = sdd::kPathsPerTask;  // paths per warp task (sdd_set_mc_config)
    int nsm = 1;
    bool fp64 = true;
    int acc_mode = sdd::kAcc64;
    int64_t step = 0;
    double t_monitor = 0.0;         // monitor time when monitor_time_fixed (M^kP sub-steps)
    bool monitor_time_fixed = false;
    bool have_est = false;
    // monitor
    int mon_kind = 0;
    int n_params = 0;
    double mon_params[64] = {0};
    // device: mesh and monitor
    double *x = nullptr, *y = nullptr, *xn = nullptr, *yn = nullptr;
    double *om64 = nullptr, *wxi64 = nullptr, *weta64 = nullptr, *omega_nodal = nullptr;
    void *mon = nullptr, *disp = nullptr;
    int2* nodes = nullptr;
    double* shift = nullptr;
    // interface sampling (iface_stride > 1): per node -1 (Monte Carlo) or its rule index
    std::vector<int32_t> h_role;
    std::vector<sdd::InterpRule> h_interp;
    int n_interp = 0;
    int32_t* iface_role = nullptr;
    sdd::InterpRule* interp = nullptr;
    // device: interface MC
    double* acc = nullptr;
    int64_t *n_done = nullptr, *steps = nullptr, *paths_run = nullptr, *next_total = nullptr;
    int32_t* node_of = nullptr;
    int64_t *p_begin = nullptr, *p_count = nullptr, *task_off = nullptr;
    int32_t *n_active = nullptr, *task_counter = nullptr;
    sdd::TaskSlot* slots = nullptr;
    int64_t slot_cap = 0;
    double *est = nullptr, *se = nullptr;
    // device: solves
    double *ce64 = nullptr, *cn64 = nullptr;
    void *ce = nullptr, *cn = nullptr, *vec = nullptr;
    void* mg = nullptr;             // multigrid workspace, mg_stride bytes per subdomain
    size_t mg_stride = 0;
    std::vector<sdd::SolveItem> h_items;  // cooperative solve items (empty: one CTA per subdomain)
    sdd::SolveItem* solve_items = nullptr;
    int32_t *st_iters = nullptr, *st_outer = nullptr, *st_ok = nullptr;
    double* st_res = nullptr;
    double* quality = nullptr;      // (nx-1)(ny-1) cell qualities + 2 stats
    int32_t* bad = nullptr;         // set by the monitor preparation on invalid monitor or mesh
    double* bnd64 = nullptr;        // moving boundary: new tangential boundary coordinates (FP64)
    void* bnd = nullptr;            //   the same in the path precision
    double* bnd_scratch = nullptr;  //   tridiagonal sweeps
    // host
    int32_t* h_n_active = nullptr;  // pinned: [0] active nodes, [1] invalid-input flag, [2..] round counts
    cudaEvent_t count_ev[sdd::kRoundsAhead + 1] = {};  // after the copies of the round counts
    sdd_stats stats{};
    std::vector<void*> allocs;
    size_t dev_bytes = 0;          // device bytes held (allocation granularity included)
    std::vector<cudaEvent_t> ev;  // start/stop pairs around path-kernel launches
    cudaEvent_t solve_ev[2] = {nullptr, nullptr};  // around the subdomain-solve launches
    int64_t launches = 0;         // kernels launched since creation

    template <typename P>
    cudaError_t dalloc(P** p, size_t bytes)
    {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, bytes < 16 ? 16 : bytes);
        if (e == cudaSuccess) {
            allocs.push_back(v);
            *p = static_cast<P*>(v);
        }
        return e;
    }
    ~sdd_problem()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaEvent_t e : count_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : solve_ev)
            if (e) cudaEventDestroy(e);
        for (void* v : allocs) cudaFree(v);
        if (h_n_active) cudaFreeHost(h_n_active);
    }
};

// Task sizes a problem or batch may use (sdd_set_mc_config).
inline bool sdd_valid_task_paths(int t) { return t == 1024 || t == 2048 || t == 4096; }

// Sets the calling thread's sdd_last_error message and returns s.
sdd_status sdd_fail(sdd_status s, const char* msg);

// Parameter checks of sdd_create_problem (sets the last error).
sdd_status sdd_validate_params(const sdd_params* P);
// Interface nodes (i, j) of a grid split, in node-id order (as sdd_interface_layout).
void sdd_layout(int nx, int ny, int px, int py, int periodic, std::vector<int32_t>& ij);
// Device bytes sdd_alloc_problem takes for these parameters.
size_t sdd_problem_device_bytes(const sdd_params& prm, bool with_mc);
// Allocates a problem's device arrays (with_mc: also its own interface MC state), uploads its
// interface nodes and zeroes the solver vectors, all on `stream` (synchronised).  The mesh and
// monitor are left for the caller to fill.
sdd_status sdd_alloc_problem(const sdd_params& prm, cudaStream_t stream, bool with_mc, sdd_problem** out);
// Host check of a Dirichlet mesh's boundary: (Lx xi, Ly eta) within 1e-12 (Lx + Ly).
bool sdd_boundary_ok(const sdd_params& prm, const double* hx, const double* hy);

// Path-kernel record of a problem at its current step.
template <typename T>
inline sdd::McProblem<T> mc_problem(const sdd_problem* p)
{
    sdd::McProblem<T> R{};
    R.mon = static_cast<const sdd::Mon4<T>*>(p->mon);
    R.disp = static_cast<const sdd::Disp2<T>*>(p->disp);
    R.nodes = p->nodes;
    R.nx = p->prm.nx; R.ny = p->prm.ny; R.periodic = p->prm.periodic; R.form = p->prm.form;
    R.K = p->prm.substeps; R.bicubic = p->prm.bicubic; R.bb = p->prm.bb_test;
    const T ds = (T)p->prm.dt / (T)p->prm.substeps;
    R.cb = ds / (T)p->prm.tau;
    R.Lx = (T)p->prm.Lx; R.Ly = (T)p->prm.Ly;
    R.key0 = (uint32_t)(p->prm.seed & 0xFFFFFFFFu);
    R.key1 = (uint32_t)(p->prm.seed >> 32);
    sdd::philox_round_keys(p->prm.seed, R.rk);
    sdd::set_grid_consts(R);
    R.tstep = (uint32_t)p->step;
    R.node_offset = 0;
    R.bnd = p->prm.moving_boundary ? static_cast<const T*>(p->bnd) : nullptr;
    return R;
}

