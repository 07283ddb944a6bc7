// Batched stepping of independent SDD problems (sdd_batch_*, declared in include/sdd.h).
//
// Many mesh problems of uneven grid and subdomain counts advance one alternating step
// together: per problem, the monitor preparation and the Dirichlet-data scatter; then ONE
// persistent path-kernel launch per round serves the interface nodes of every problem (the
// round plan runs over the concatenated node list, every task carries its problem), and ONE
// launch solves every subdomain of every problem (one CTA per (problem, subdomain)).
//
// A problem's results do not depend on its batch: its paths use its own seed and local node
// ids in the Philox counter, its nodes follow their own chunk schedule, and every sum is a
// fixed-order reduction over its own tasks -- the meshes are bitwise those of stepping each
// problem alone.
//
// Per-step inputs that change between steps (time-step index, time) are read from device
// records refreshed from pinned host memory at the start of each step, and the new mesh is
// copied into the current one instead of swapping pointers, so a fixed-N step is one fixed
// launch sequence: with use_graph it is captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sdd.h"
#include "sdd_internal.cuh"
#include "sdd_problem.cuh"

using namespace sdd;

namespace {

constexpr int kSlotsPerNode = kTasksPerRound;  // task slots per node: one round's tasks
constexpr int kMaxRounds = 4096;

}  // namespace

struct sdd_batch {
    std::vector<sdd_problem*> probs;
    cudaStream_t stream = nullptr;
    bool fp64 = false;
    int acc_mode = kAcc64;
    bool use_graph = false;
    int n = 0;
    int M = 0;                       // interface nodes of all problems
    int total_subs = 0;
    std::vector<int32_t> node_off, sub_off;
    int mc_grid = 1;
    int tpb = 256;                   // path-kernel threads per block (sdd_batch_tune)
    int bps = 0;                     // resident path-kernel blocks per SM (0: the register limit)
    int max_bps = 1;                 // the register limit at tpb
    int task_paths = kPathsPerTask;  // paths per warp task, shared by every problem
    int nsm = 1;
    // device: concatenated node arrays and round plan
    int32_t* node_prob = nullptr;
    int32_t* node_role = nullptr;    // concatenated sampling roles (null: every node by Monte Carlo)
    double *shift = nullptr, *acc = nullptr, *est = nullptr, *se = nullptr;
    int64_t *n_done = nullptr, *steps = nullptr, *paths_run = nullptr, *next_total = nullptr;
    int64_t *p_begin = nullptr, *p_count = nullptr, *task_off = nullptr;
    int32_t *node_of = nullptr, *n_active = nullptr, *task_counter = nullptr;
    TaskSlot* slots = nullptr;
    // device records refreshed every step, and their pinned host sources
    void* mcprob_dev = nullptr;
    void* mcprob_host = nullptr;
    SolveParams* solve_dev = nullptr;
    SolveParams* solve_host = nullptr;
    double* t_dev = nullptr;
    double* t_host = nullptr;
    int32_t* sub_off_dev = nullptr;
    int2* order_dev = nullptr;       // solve CTAs: (problem, subdomain), largest subdomains first
    SolveItem* items_dev = nullptr;  // cooperative solve items (n_items > 0: large subdomains present)
    int n_items = 0;
    // batched per-problem launches: records (refreshed every step) and per-problem block offsets
    BatchRec* rec_dev = nullptr;
    BatchRec* rec_host = nullptr;
    int32_t* blk_off_dev = nullptr;
    int total_blocks = 0;
    bool any_moving = false;
    int mc_mode = -1;            // problem switches shared by every problem (launch_mc's batch_mode), or -1
    int32_t* h_n_active = nullptr;
    // graph
    cudaGraphExec_t graph = nullptr;
    std::vector<const double*> graph_x;  // mesh pointers the graph was recorded with
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t sev0 = nullptr, sev1 = nullptr;  // around the batched face + solve launches
    cudaEvent_t count_ev[kRoundsAhead + 1] = {};  // after the round-count copies to h_n_active[2..]
    int64_t launches = 0;
    int64_t launches_per_step = 0;
    int32_t rounds_last = 0;
    double step_ms_last = 0.0;
    std::vector<void*> allocs;
    std::vector<void*> host_allocs;

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
    template <typename P>
    cudaError_t halloc(P** p, size_t bytes)
    {
        void* v = nullptr;
        cudaError_t e = cudaHostAlloc(&v, bytes < 16 ? 16 : bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) {
            host_allocs.push_back(v);
            *p = static_cast<P*>(v);
        }
        return e;
    }
    ~sdd_batch()
    {
        if (graph) cudaGraphExecDestroy(graph);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (sev0) cudaEventDestroy(sev0);
        if (sev1) cudaEventDestroy(sev1);
        for (cudaEvent_t c : count_ev)
            if (c) cudaEventDestroy(c);
        for (void* v : allocs) cudaFree(v);
        for (void* v : host_allocs) cudaFreeHost(v);
    }
};

namespace {

#define B_CK(call)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            const std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);     \
            return sdd_fail(e_ == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA,  \
                            m_.c_str());                                                   \
        }                                                                                  \
    } while (0)

SolveParams solve_params(const sdd_problem* p)
{
    SolveParams S{};
    S.nx = p->prm.nx; S.ny = p->prm.ny; S.px = p->prm.px; S.py = p->prm.py; S.form = p->prm.form;
    S.r = p->prm.dt / p->prm.tau; S.rtol = p->prm.solve_rtol; S.max_iter = p->prm.solve_max_iter;
    S.scheme = p->prm.subdomain_scheme;
    S.fe_max_substeps = p->prm.fe_max_substeps > 0 ? p->prm.fe_max_substeps : (1 << 16);
    S.om64 = p->om64; S.xcur = p->x; S.ycur = p->y; S.xnew = p->xn; S.ynew = p->yn;
    S.ce64 = p->ce64; S.cn64 = p->cn64; S.ce = p->ce; S.cn = p->cn; S.vec = p->vec;
    S.mg = p->mg; S.mg_stride = p->mg_stride;
    S.stat_iters = p->st_iters; S.stat_outer = p->st_outer; S.stat_ok = p->st_ok; S.stat_res = p->st_res;
    return S;
}

// Host copies of the per-step records (call with no step of this batch in flight).
void refresh_records(sdd_batch* b)
{
    for (int i = 0; i < b->n; ++i) {
        const sdd_problem* p = b->probs[i];
        if (b->fp64) {
            McProblem<double> R = mc_problem<double>(p);
            R.node_offset = b->node_off[i];
            static_cast<McProblem<double>*>(b->mcprob_host)[i] = R;
        } else {
            McProblem<float> R = mc_problem<float>(p);
            R.node_offset = b->node_off[i];
            static_cast<McProblem<float>*>(b->mcprob_host)[i] = R;
        }
        b->solve_host[i] = solve_params(p);
        b->t_host[i] = p->prm.t0 + (double)p->step * p->prm.dt;
        BatchRec& r = b->rec_host[i];
        r = BatchRec{};
        PrepParams& P = r.prep;
        P.nx = p->prm.nx; P.ny = p->prm.ny; P.periodic = p->prm.periodic;
        P.kind = p->mon_kind; P.n_params = p->n_params; P.precision = p->prm.precision;
        P.Lx = p->prm.Lx; P.Ly = p->prm.Ly; P.t = 0.0; P.t_dev = b->t_dev + i;
        P.x = p->x; P.y = p->y; P.omega_in = p->omega_nodal;
        memcpy(P.params, p->mon_params, sizeof(P.params));
        P.om64 = p->om64; P.wxi64 = p->wxi64; P.weta64 = p->weta64; P.mon = p->mon; P.disp = p->disp;
        P.bad = p->bad;
        P.moving_boundary = p->prm.moving_boundary; P.form = p->prm.form; P.r = p->prm.dt / p->prm.tau;
        P.bnd64 = p->bnd64; P.bnd = p->bnd; P.bnd_scratch = p->bnd_scratch;
        r.nodes = p->nodes;
        r.node_offset = b->node_off[i];
        r.xnew = p->xn;
        r.ynew = p->yn;
    }
}

template <typename T>
sdd_status launch_batch_mc(sdd_batch* b)
{
    McParams<T> P{};
    P.probs = static_cast<const McProblem<T>*>(b->mcprob_dev);
    P.node_prob = b->node_prob;
    P.shift = b->shift;
    P.node_of = b->node_of; P.p_begin = b->p_begin; P.p_count = b->p_count; P.task_off = b->task_off;
    P.n_active = b->n_active; P.task_counter = b->task_counter; P.slots = b->slots;
    P.task_paths = b->task_paths;
    B_CK(launch_mc<T>(P, b->acc_mode, false, true, b->mc_grid, b->stream, b->tpb, b->mc_mode));
    return SDD_OK;
}

// Path-kernel block size and the persistent grid: bps resident blocks on every SM (0: all the
// kernel's registers allow at that block size).
void set_block_size(sdd_batch* b, int tpb, int bps = 0)
{
    b->tpb = tpb;
    b->max_bps = b->fp64 ? mc_max_blocks_per_sm<double>(b->acc_mode, false, true, tpb)
                         : mc_max_blocks_per_sm<float>(b->acc_mode, false, true, tpb);
    b->bps = bps > 0 && bps < b->max_bps ? bps : 0;
    b->mc_grid = b->nsm * (b->bps > 0 ? b->bps : b->max_bps);
}

// The launches of one step.  `capturing`: only fixed-N work (no host round trip).  first_plan:
// stop after planning the first Monte Carlo round (used to time the path kernel).
sdd_status record_step(sdd_batch* b, bool first_plan = false)
{
    const size_t rec = b->fp64 ? sizeof(McProblem<double>) : sizeof(McProblem<float>);
    int64_t launches = 0;
    B_CK(cudaMemcpyAsync(b->mcprob_dev, b->mcprob_host, rec * b->n, cudaMemcpyHostToDevice, b->stream));
    B_CK(cudaMemcpyAsync(b->solve_dev, b->solve_host, sizeof(SolveParams) * b->n, cudaMemcpyHostToDevice,
                         b->stream));
    B_CK(cudaMemcpyAsync(b->t_dev, b->t_host, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream));
    B_CK(cudaMemcpyAsync(b->rec_dev, b->rec_host, sizeof(BatchRec) * b->n, cudaMemcpyHostToDevice, b->stream));
    // monitor, packing and moving boundary of every problem, then the estimator shifts: one launch each
    B_CK(launch_prep_batch(b->rec_dev, b->blk_off_dev, b->n, b->total_blocks, b->fp64, b->any_moving, b->stream));
    launches += 2 + (b->any_moving ? 1 : 0);
    if (b->M > 0) {
        B_CK(launch_shift_batch(b->rec_dev, b->node_prob, b->M, b->shift, b->stream));
        launches += 1;
    }
    if (b->M > 0) {
        const sdd_params& q = b->probs[0]->prm;
        const bool adaptive = q.se_target > 0;
        const int64_t n0 = q.paths_per_node;
        const int64_t maxp = adaptive ? q.max_paths_per_node : n0;
        B_CK(launch_mc_init(b->M, n0, maxp, b->acc, b->n_done, b->steps, b->paths_run, b->next_total,
                            b->stream, b->node_role));
        launches += 1;
        PlanParams PP{};
        PP.M = b->M; PP.n_done = b->n_done; PP.next_total = b->next_total; PP.node_of = b->node_of;
        PP.p_begin = b->p_begin; PP.p_count = b->p_count; PP.task_off = b->task_off;
        PP.n_active = b->n_active; PP.task_counter = b->task_counter;
        PP.task_paths = b->task_paths;
        ReduceParams RP{};
        RP.node_of = b->node_of; RP.p_count = b->p_count; RP.task_off = b->task_off; RP.n_active = b->n_active;
        RP.slots = b->slots; RP.shift = b->shift; RP.acc = b->acc; RP.n_done = b->n_done; RP.steps = b->steps;
        RP.paths_run = b->paths_run; RP.next_total = b->next_total;
        RP.se_target = adaptive ? q.se_target : 0.0; RP.max_paths = maxp;
        if (first_plan) {
            B_CK(launch_plan(PP, b->stream));
            return SDD_OK;
        }
        int32_t rounds = 0;
        if (!adaptive) {
            const int64_t chunk = (int64_t)kTasksPerRound * b->task_paths;
            const int64_t nr = (n0 + chunk - 1) / chunk;
            for (int64_t r = 0; r < nr; ++r) {
                B_CK(launch_plan(PP, b->stream));
                const sdd_status s = b->fp64 ? launch_batch_mc<double>(b) : launch_batch_mc<float>(b);
                if (s != SDD_OK) return s;
                B_CK(launch_reduce(RP, b->M, b->stream));
                launches += 3;
                rounds += 1;
            }
        } else {
            // kRoundsAhead rounds ahead of the host's decision, as for a single problem: rounds
            // queued after the last one with work find no pending node and change nothing
            int queued = 0;
            for (int r = 0; r < kMaxRounds; ++r) {
                for (; queued < kMaxRounds && queued <= r + kRoundsAhead; ++queued) {
                    const int slot = queued % (kRoundsAhead + 1);
                    B_CK(launch_plan(PP, b->stream));
                    B_CK(cudaMemcpyAsync(b->h_n_active + 2 + slot, b->n_active, 4, cudaMemcpyDeviceToHost,
                                         b->stream));
                    B_CK(cudaEventRecord(b->count_ev[slot], b->stream));
                    const sdd_status s = b->fp64 ? launch_batch_mc<double>(b) : launch_batch_mc<float>(b);
                    if (s != SDD_OK) return s;
                    B_CK(launch_reduce(RP, b->M, b->stream));
                    launches += 3;
                }
                const int slot = r % (kRoundsAhead + 1);
                B_CK(cudaEventSynchronize(b->count_ev[slot]));
                if (b->h_n_active[2 + slot] == 0) break;
                rounds = r + 1;
            }
        }
        b->rounds_last = rounds;
        B_CK(launch_output(b->M, b->acc, b->n_done, b->shift, b->est, b->se, b->stream));
        launches += 1;
        for (int i = 0; i < b->n; ++i) {
            sdd_problem* p = b->probs[i];
            if (p->n_interp == 0) continue;
            const size_t o = (size_t)b->node_off[i];
            B_CK(launch_interp(p->interp, p->n_interp, b->est + 2 * o, b->se + 2 * o, b->stream));
            launches += 1;
        }
    }
    const bool fp64_inner = b->fp64;
    // Dirichlet rims and interface estimates into every new mesh, then the face coefficients
    B_CK(launch_scatter_batch(b->rec_dev, b->blk_off_dev, b->n, b->total_blocks, b->node_prob, b->M, b->est,
                              b->stream));
    launches += 1 + (b->M > 0 ? 1 : 0);
    B_CK(launch_faces_batch(b->solve_dev, b->blk_off_dev, b->n, b->total_blocks, fp64_inner, b->stream));
    launches += 1;
    bool any_be = false, any_fe = false;
    for (const sdd_problem* p : b->probs) {
        any_be = any_be || p->prm.subdomain_scheme == 0;
        any_fe = any_fe || p->prm.subdomain_scheme == 1;
    }
    B_CK(cudaEventRecord(b->sev0, b->stream));
    if (b->n_items > 0) {
        B_CK(launch_solve_batch_items(b->solve_dev, b->items_dev, b->n_items, fp64_inner, b->stream));
        if (any_fe)
            B_CK(launch_solve_batch(b->solve_dev, b->sub_off_dev, b->n, b->total_subs, fp64_inner, b->stream,
                                    false, true, b->order_dev));
    } else {
        B_CK(launch_solve_batch(b->solve_dev, b->sub_off_dev, b->n, b->total_subs, fp64_inner, b->stream, any_be,
                                any_fe, b->order_dev));
    }
    B_CK(cudaEventRecord(b->sev1, b->stream));
    launches += (any_be ? 1 : 0) + (any_fe ? 1 : 0);
    B_CK(launch_copy_back_batch(b->rec_dev, b->blk_off_dev, b->n, b->total_blocks, b->stream));
    launches += 1;
    b->launches_per_step = launches;
    return SDD_OK;
}

}  // namespace

extern "C" {

sdd_status sdd_batch_create(sdd_problem* const* problems, int32_t n, void* stream, int32_t use_graph,
                            sdd_batch** out)
{
    if (!out) return sdd_fail(SDD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!problems || n < 1) return sdd_fail(SDD_ERR_INVALID_ARG, "need at least one problem");
    if (use_graph != 0 && use_graph != 1) return sdd_fail(SDD_ERR_INVALID_ARG, "use_graph must be 0 or 1");
    for (int i = 0; i < n; ++i)
        if (!problems[i]) return sdd_fail(SDD_ERR_INVALID_ARG, "NULL problem");
    const sdd_params& q = problems[0]->prm;
    for (int i = 1; i < n; ++i) {
        const sdd_params& r = problems[i]->prm;
        if (r.precision != q.precision || r.se_target != q.se_target || r.paths_per_node != q.paths_per_node ||
            (q.se_target > 0 && r.max_paths_per_node != q.max_paths_per_node) ||
            problems[i]->task_paths != problems[0]->task_paths)
            return sdd_fail(SDD_ERR_INVALID_ARG,
                            "batched problems must share precision, se_target, path counts and paths_per_task");
        for (int k = 0; k < i; ++k)
            if (problems[k] == problems[i]) return sdd_fail(SDD_ERR_INVALID_ARG, "a problem appears twice");
    }
    if (use_graph && (q.se_target > 0 || !stream))
        return sdd_fail(SDD_ERR_INVALID_ARG, "graph mode needs fixed N and a non-NULL stream");
    int64_t m_total = 0;
    for (int i = 0; i < n; ++i) m_total += problems[i]->M;
    if (m_total >= ((int64_t)1 << 23))  // a round's tasks (up to kSlotsPerNode per node) fit in an int
        return sdd_fail(SDD_ERR_INVALID_ARG, "the batch's interface nodes must number below 2^23");
    sdd_batch* b = new sdd_batch();
    b->probs.assign(problems, problems + n);
    b->n = n;
    b->stream = static_cast<cudaStream_t>(stream);
    b->fp64 = q.precision == SDD_FP64;
    b->acc_mode = q.precision == SDD_FP32_KAHAN ? kAccKahan32 : kAcc64;
    b->use_graph = use_graph != 0;
    b->task_paths = problems[0]->task_paths;
    std::vector<int32_t> node_prob, node_role;
    bool sampled_any = false;
    b->sub_off.push_back(0);
    for (int i = 0; i < n; ++i) {
        b->node_off.push_back(b->M);
        b->M += problems[i]->M;
        node_prob.insert(node_prob.end(), problems[i]->M, i);
        node_role.insert(node_role.end(), problems[i]->h_role.begin(), problems[i]->h_role.end());
        sampled_any = sampled_any || problems[i]->n_interp > 0;
        b->total_subs += problems[i]->prm.px * problems[i]->prm.py;
        b->sub_off.push_back(b->total_subs);
    }
    const size_t M = (size_t)b->M + 1;
    const size_t rec = b->fp64 ? sizeof(McProblem<double>) : sizeof(McProblem<float>);
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) if (e == cudaSuccess) e = b->dalloc(&(ptr), (bytes))
#define HALLOC(ptr, bytes) if (e == cudaSuccess) e = b->halloc(&(ptr), (bytes))
    ALLOC(b->node_prob, M * 4); ALLOC(b->shift, M * 16); ALLOC(b->acc, M * 32); ALLOC(b->est, M * 16);
    ALLOC(b->se, M * 16); ALLOC(b->n_done, M * 8); ALLOC(b->steps, M * 8); ALLOC(b->paths_run, M * 8);
    ALLOC(b->next_total, M * 8); ALLOC(b->p_begin, M * 8); ALLOC(b->p_count, M * 8);
    ALLOC(b->task_off, (M + 1) * 8); ALLOC(b->node_of, M * 4); ALLOC(b->n_active, 16);
    ALLOC(b->task_counter, 16); ALLOC(b->slots, M * kSlotsPerNode * sizeof(TaskSlot));
    ALLOC(b->mcprob_dev, rec * n); ALLOC(b->solve_dev, sizeof(SolveParams) * n); ALLOC(b->t_dev, 8 * n);
    ALLOC(b->sub_off_dev, 4 * (n + 1));
    ALLOC(b->rec_dev, sizeof(BatchRec) * n); ALLOC(b->blk_off_dev, 4 * (n + 1));
    ALLOC(b->order_dev, sizeof(int2) * (size_t)(b->total_subs > 0 ? b->total_subs : 1));
    if (sampled_any) ALLOC(b->node_role, M * 4);
    HALLOC(b->mcprob_host, rec * n); HALLOC(b->solve_host, sizeof(SolveParams) * n); HALLOC(b->t_host, 8 * n);
    HALLOC(b->h_n_active, 32); HALLOC(b->rec_host, sizeof(BatchRec) * n);
#undef ALLOC
#undef HALLOC
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&b->sev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->sev1);
    for (int k = 0; k <= kRoundsAhead && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&b->count_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess && b->M > 0)
        e = cudaMemcpy(b->node_prob, node_prob.data(), 4 * (size_t)b->M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->sub_off_dev, b->sub_off.data(), 4 * (size_t)(n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<int32_t> blk_off(1, 0);
        for (int i = 0; i < n; ++i) {
            blk_off.push_back(blk_off.back() + batch_blocks((long)problems[i]->prm.nx * problems[i]->prm.ny));
            b->any_moving = b->any_moving || (problems[i]->prm.moving_boundary && !problems[i]->prm.periodic);
        }
        b->total_blocks = blk_off.back();
        e = cudaMemcpy(b->blk_off_dev, blk_off.data(), 4 * (size_t)(n + 1), cudaMemcpyHostToDevice);
        // the problem switches, when every problem shares them (the path kernel then has them compiled in)
        for (int i = 0; i < n; ++i) {
            const sdd_params& q = problems[i]->prm;
            const int mode = (q.periodic ? 1 : 0) | (q.form ? 2 : 0) | (q.bb_test ? 4 : 0);
            b->mc_mode = i == 0 ? mode : (b->mc_mode == mode ? mode : -1);
        }
    }
    if (e == cudaSuccess && b->total_subs > 0) {
        // longest-first: subdomains by interior size, descending (ties in problem, subdomain order)
        std::vector<std::pair<int64_t, int2>> subs;
        for (int i = 0; i < n; ++i) {
            const sdd_params& q = problems[i]->prm;
            for (int k = 0; k < q.px * q.py; ++k) {
                const int I = k % q.px, J = k / q.px;
                const int64_t wi = split_line(I + 1, q.nx, q.px) - split_line(I, q.nx, q.px) - 1;
                const int64_t wj = split_line(J + 1, q.ny, q.py) - split_line(J, q.ny, q.py) - 1;
                subs.push_back({wi * wj, make_int2(i, k)});
            }
        }
        std::stable_sort(subs.begin(), subs.end(), [](const std::pair<int64_t, int2>& a,
                                                      const std::pair<int64_t, int2>& c) { return a.first > c.first; });
        std::vector<int2> order;
        for (const auto& v : subs) order.push_back(v.second);
        e = cudaMemcpy(b->order_dev, order.data(), sizeof(int2) * order.size(), cudaMemcpyHostToDevice);
        // backward-Euler subdomains only: forward-Euler problems run in their own kernel
        std::vector<std::pair<int64_t, int2>> be;
        for (const auto& v : subs)
            if (problems[v.second.x]->prm.subdomain_scheme == 0) be.push_back(v);
        const std::vector<SolveItem> items = solve_items(be);
        if (e == cudaSuccess && !items.empty()) {
            e = b->dalloc(&b->items_dev, sizeof(SolveItem) * items.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(b->items_dev, items.data(), sizeof(SolveItem) * items.size(), cudaMemcpyHostToDevice);
            b->n_items = (int)items.size();
        }
    }
    if (e == cudaSuccess && sampled_any && b->M > 0)
        e = cudaMemcpy(b->node_role, node_role.data(), 4 * (size_t)b->M, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const std::string m = std::string("batch allocation failed: ") + cudaGetErrorString(e);
        delete b;
        return sdd_fail(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, m.c_str());
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    set_block_size(b, 256);
    *out = b;
    return SDD_OK;
}

void sdd_batch_destroy(sdd_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    delete b;
}

sdd_status sdd_batch_step(sdd_batch* b)
{
    if (!b) return sdd_fail(SDD_ERR_INVALID_ARG, "batch is NULL");
    const TraceRange trace("sdd_batch_step");
    for (sdd_problem* p : b->probs) B_CK(cudaStreamSynchronize(p->stream));
    B_CK(cudaStreamSynchronize(b->stream));  // no step of this batch in flight: safe to refresh records
    refresh_records(b);
    B_CK(cudaEventRecord(b->ev0, b->stream));
    if (b->use_graph) {
        bool stale = !b->graph || b->graph_x.size() != b->probs.size();
        for (size_t i = 0; !stale && i < b->probs.size(); ++i) stale = b->graph_x[i] != b->probs[i]->x;
        if (stale) {
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            B_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            const sdd_status s = record_step(b);
            const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (s != SDD_OK) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            if (ce != cudaSuccess) return sdd_fail(SDD_ERR_CUDA, cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) return sdd_fail(SDD_ERR_CUDA, cudaGetErrorString(ie));
            b->graph_x.clear();
            for (sdd_problem* p : b->probs) b->graph_x.push_back(p->x);
        }
        B_CK(cudaGraphLaunch(b->graph, b->stream));
    } else {
        const sdd_status s = record_step(b);
        if (s != SDD_OK) return s;
    }
    B_CK(cudaEventRecord(b->ev1, b->stream));
    b->launches += b->launches_per_step;
    for (sdd_problem* p : b->probs) {
        p->step += 1;
        p->have_est = false;
        p->stats.step_index = (int32_t)p->step;
        p->stats.t = p->prm.t0 + (double)p->step * p->prm.dt;
    }
    return SDD_OK;
}

sdd_status sdd_batch_tune(sdd_batch* b, int32_t threads_per_block, int32_t* chosen)
{
    if (!b) return sdd_fail(SDD_ERR_INVALID_ARG, "batch is NULL");
    if (threads_per_block != 0 && threads_per_block != 128 && threads_per_block != 256 && threads_per_block != 512)
        return sdd_fail(SDD_ERR_INVALID_ARG, "threads_per_block must be 0, 128, 256 or 512");
    const TraceRange trace("sdd_batch_tune");
    for (sdd_problem* p : b->probs) B_CK(cudaStreamSynchronize(p->stream));
    B_CK(cudaStreamSynchronize(b->stream));
    int pick = threads_per_block;
    if (pick == 0 && b->M == 0) pick = b->tpb;
    if (pick == 0) {
        // the next step's first round, up to its plan; then one path-kernel launch per candidate
        // on that plan, into the scratch task slots (no problem's state changes: the next step
        // prepares, initialises and plans again)
        refresh_records(b);
        sdd_status st = record_step(b, true);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t ce = cudaSuccess;
        if (st == SDD_OK) ce = cudaEventCreate(&e0);
        if (st == SDD_OK && ce == cudaSuccess) ce = cudaEventCreate(&e1);
        float best = 0.f;
        const int cand[3] = {128, 256, 512};
        for (int k = 0; k < 3 && st == SDD_OK && ce == cudaSuccess; ++k) {
            set_block_size(b, cand[k]);
            ce = cudaMemsetAsync(b->task_counter, 0, sizeof(int32_t), b->stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, b->stream);
            if (ce != cudaSuccess) break;
            st = b->fp64 ? launch_batch_mc<double>(b) : launch_batch_mc<float>(b);
            if (st != SDD_OK) break;
            ce = cudaEventRecord(e1, b->stream);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce == cudaSuccess && (pick == 0 || ms < best)) {
                best = ms;
                pick = cand[k];
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st != SDD_OK) return st;
        if (ce != cudaSuccess) return sdd_fail(SDD_ERR_CUDA, cudaGetErrorString(ce));
    }
    set_block_size(b, pick);
    if (b->graph) {  // recorded with the previous size
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (chosen) *chosen = b->tpb;
    return SDD_OK;
}

sdd_status sdd_batch_get_mc_config(sdd_batch* b, sdd_mc_config* out)
{
    if (!b || !out) return sdd_fail(SDD_ERR_INVALID_ARG, "NULL argument");
    out->threads_per_block = b->tpb;
    out->blocks_per_sm = b->bps > 0 ? b->bps : b->max_bps;
    out->paths_per_task = b->task_paths;
    out->max_blocks_per_sm = b->max_bps;
    return SDD_OK;
}

namespace {

// Applies a validated configuration (tpb, bps, task size) to the batch and its problems.
void apply_mc_config(sdd_batch* b, int tpb, int bps, int task_paths)
{
    set_block_size(b, tpb, bps);
    b->task_paths = task_paths;
    for (sdd_problem* p : b->probs) p->task_paths = task_paths;
    if (b->graph) {  // recorded with the previous configuration
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

}  // namespace

sdd_status sdd_batch_set_mc_config(sdd_batch* b, const sdd_mc_config* c)
{
    if (!b || !c) return sdd_fail(SDD_ERR_INVALID_ARG, "NULL argument");
    const int tpb = c->threads_per_block ? c->threads_per_block : b->tpb;
    if (tpb != 128 && tpb != 256 && tpb != 512)
        return sdd_fail(SDD_ERR_INVALID_ARG, "threads_per_block must be 0, 128, 256 or 512");
    const int max_bps = b->fp64 ? mc_max_blocks_per_sm<double>(b->acc_mode, false, true, tpb)
                                : mc_max_blocks_per_sm<float>(b->acc_mode, false, true, tpb);
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > max_bps)
        return sdd_fail(SDD_ERR_INVALID_ARG, "blocks_per_sm must be in [0, the limit at threads_per_block]");
    if (c->paths_per_task != 0 && !sdd_valid_task_paths(c->paths_per_task))
        return sdd_fail(SDD_ERR_INVALID_ARG, "paths_per_task must be 1024, 2048 or 4096");
    for (sdd_problem* p : b->probs) B_CK(cudaStreamSynchronize(p->stream));
    B_CK(cudaStreamSynchronize(b->stream));
    apply_mc_config(b, tpb, c->blocks_per_sm, c->paths_per_task ? c->paths_per_task : b->task_paths);
    return SDD_OK;
}

sdd_status sdd_batch_tune_mc(sdd_batch* b, int32_t tune_paths_per_task, sdd_mc_config* chosen)
{
    if (!b) return sdd_fail(SDD_ERR_INVALID_ARG, "batch is NULL");
    if (tune_paths_per_task != 0 && tune_paths_per_task != 1)
        return sdd_fail(SDD_ERR_INVALID_ARG, "tune_paths_per_task must be 0 or 1");
    const TraceRange trace("sdd_batch_tune_mc");
    for (sdd_problem* p : b->probs) B_CK(cudaStreamSynchronize(p->stream));
    B_CK(cudaStreamSynchronize(b->stream));
    if (b->M > 0) {
        // the next step's first round, up to its plan (no problem's state changes: the next step
        // prepares, initialises and plans again); then per candidate a plan at its task size and
        // one timed path-kernel launch (the faster of two) into the scratch task slots
        const int tpb0 = b->tpb, bps0 = b->bps, tp0 = b->task_paths;
        refresh_records(b);
        sdd_status st = record_step(b, true);
        const sdd_params& q = b->probs[0]->prm;
        const int64_t n0 = q.paths_per_node;
        PlanParams PP{};
        PP.M = b->M; PP.n_done = b->n_done; PP.next_total = b->next_total; PP.node_of = b->node_of;
        PP.p_begin = b->p_begin; PP.p_count = b->p_count; PP.task_off = b->task_off;
        PP.n_active = b->n_active; PP.task_counter = b->task_counter;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t ce = cudaSuccess;
        if (st == SDD_OK) ce = cudaEventCreate(&e0);
        if (st == SDD_OK && ce == cudaSuccess) ce = cudaEventCreate(&e1);
        const int tps[3] = {1024, 2048, 4096}, tpbs[3] = {128, 256, 512};
        const int nt = tune_paths_per_task ? 3 : 1;
        double best = -1.0;
        int best_tpb = tpb0, best_bps = bps0, best_t = tp0;
        for (int a = 0; a < nt && st == SDD_OK && ce == cudaSuccess; ++a) {
            const int T = tune_paths_per_task ? tps[a] : tp0;
            const int64_t round = n0 < (int64_t)kTasksPerRound * T ? n0 : (int64_t)kTasksPerRound * T;
            PP.task_paths = T;
            b->task_paths = T;  // read by launch_batch_mc; restored or replaced below
            for (int k = 0; k < 3 && st == SDD_OK && ce == cudaSuccess; ++k) {
                set_block_size(b, tpbs[k]);
                const int max_bps = b->max_bps;
                for (int bps = 1; bps <= max_bps && st == SDD_OK && ce == cudaSuccess; ++bps) {
                    set_block_size(b, tpbs[k], bps);
                    float ms_min = 0.f;
                    for (int rep = 0; rep < 2 && st == SDD_OK && ce == cudaSuccess; ++rep) {
                        ce = launch_plan(PP, b->stream);
                        if (ce == cudaSuccess) ce = cudaEventRecord(e0, b->stream);
                        if (ce != cudaSuccess) break;
                        st = b->fp64 ? launch_batch_mc<double>(b) : launch_batch_mc<float>(b);
                        if (st != SDD_OK) break;
                        ce = cudaEventRecord(e1, b->stream);
                        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                        if (ce == cudaSuccess && (rep == 0 || ms < ms_min)) ms_min = ms;
                        b->launches += 2;
                    }
                    const double per_path = (double)ms_min / (double)round;
                    if (st == SDD_OK && ce == cudaSuccess && (best < 0 || per_path < best)) {
                        best = per_path;
                        best_tpb = tpbs[k];
                        best_bps = bps;
                        best_t = T;
                    }
                }
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st != SDD_OK || ce != cudaSuccess) {
            apply_mc_config(b, tpb0, bps0, tp0);
            if (st != SDD_OK) return st;
            cudaGetLastError();
            return sdd_fail(SDD_ERR_CUDA, cudaGetErrorString(ce));
        }
        apply_mc_config(b, best_tpb, best_bps, best_t);
    }
    return chosen ? sdd_batch_get_mc_config(b, chosen) : SDD_OK;
}

sdd_status sdd_batch_get_stats(sdd_batch* b, sdd_stats* out)
{
    if (!b || !out) return sdd_fail(SDD_ERR_INVALID_ARG, "NULL argument");
    B_CK(cudaStreamSynchronize(b->stream));
    sdd_stats s{};
    s.M = b->M;
    s.step_index = b->probs[0]->stats.step_index;
    s.t = b->probs[0]->stats.t;
    s.mc_rounds = b->rounds_last;
    s.kernel_launches = b->launches;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) s.mc_kernel_ms = ms;  // whole last step
    if (cudaEventElapsedTime(&ms, b->sev0, b->sev1) == cudaSuccess) s.solve_kernel_ms = ms;  // batched solve
    cudaGetLastError();
    if (b->M > 0) {
        std::vector<int64_t> st(b->M), np(b->M);
        std::vector<double> se((size_t)2 * b->M);
        B_CK(cudaMemcpy(st.data(), b->steps, 8 * (size_t)b->M, cudaMemcpyDeviceToHost));
        B_CK(cudaMemcpy(np.data(), b->paths_run, 8 * (size_t)b->M, cudaMemcpyDeviceToHost));
        B_CK(cudaMemcpy(se.data(), b->se, 16 * (size_t)b->M, cudaMemcpyDeviceToHost));
        const double target = b->probs[0]->prm.se_target;
        for (int m = 0; m < b->M; ++m) {
            s.path_steps += st[m];
            s.paths += np[m];
            const double v = se[2 * m] > se[2 * m + 1] ? se[2 * m] : se[2 * m + 1];
            if (v > s.max_se) s.max_se = v;
            if (target > 0 && v > target) s.nodes_not_reached += 1;
        }
    }
    int invalid = 0;
    for (sdd_problem* p : b->probs) {
        int32_t flag = 0;
        B_CK(cudaMemcpy(&flag, p->bad, 4, cudaMemcpyDeviceToHost));
        invalid += flag ? 1 : 0;
        const int ns = p->prm.px * p->prm.py;
        std::vector<int32_t> it(ns), ou(ns);
        std::vector<double> rs(ns);
        B_CK(cudaMemcpy(it.data(), p->st_iters, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
        B_CK(cudaMemcpy(ou.data(), p->st_outer, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
        B_CK(cudaMemcpy(rs.data(), p->st_res, 8 * (size_t)ns, cudaMemcpyDeviceToHost));
        for (int k = 0; k < ns; ++k) {
            if (it[k] > s.solve_iters_max) s.solve_iters_max = it[k];
            if (ou[k] > s.solve_outer_max) s.solve_outer_max = ou[k];
            if (rs[k] > s.solve_rel_residual) s.solve_rel_residual = rs[k];
        }
    }
    *out = s;
    if (invalid) return sdd_fail(SDD_ERR_INVALID_ARG, "a problem's monitor is not finite and > 0 (or its mesh not finite)");
    return SDD_OK;
}

}  // extern "C"
