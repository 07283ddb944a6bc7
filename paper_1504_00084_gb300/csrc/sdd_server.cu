// Serving of one-step requests with continuous batching (sdd_server_*, declared in
// include/sdd.h).
//
// Requests arrive over time, each one alternating step (Sec. 3.6) of its own mesh problem.
// All running requests share ONE node pool: a request holds a contiguous range of pool nodes
// (its interface nodes, local id = pool index - range start), the pool carries the per-node
// sums and schedule, and every round is one persistent path-kernel launch over the pool
// followed by one reduce launch.  Between rounds the host collects finished requests, admits
// queued ones and finishes every request whose nodes have all reached the service level
// (estimates, Dirichlet scatter, subdomain solves) on a second stream while the next round
// samples the others.  Nothing about a request depends on its neighbours in the pool: the
// Philox counter uses the local node id and the request's own seed and step index, each node
// follows its own chunk schedule, and all sums are fixed-order reductions over the node's own
// tasks, so a result is bitwise that of sdd_step on the same problem alone.
//
// Host state machine of a request: QUEUED -> RUNNING (device state, pool range) -> FINISHING
// (finish work queued) -> DONE (work complete, result held) -> collected (state released to
// the per-shape cache, range and slot freed).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <deque>
#include <list>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sdd.h"
#include "sdd_internal.cuh"
#include "sdd_problem.cuh"

using namespace sdd;

namespace {

constexpr int64_t kMaxChunk = int64_t(1) << 19;  // paths per node per round (plan kernel)
constexpr int kSlotsPerNode = (int)(kMaxChunk / kPathsPerTask);
constexpr unsigned kFullMask = 0xffffffffu;

__global__ void fill_i32_kernel(int32_t* a, int64_t n, int32_t v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// Per resident slot: nodes of its pool range still scheduled for more paths (one warp a slot).
__global__ void slot_pending_kernel(const int2* range, int n_slots, const int64_t* n_done,
                                    const int64_t* next_total, int32_t* pending)
{
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= n_slots) return;
    const int2 r = range[w];
    int c = 0;
    for (int m = r.x + lane; m < r.x + r.y; m += 32) c += next_total[m] > n_done[m] ? 1 : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(kFullMask, c, off);
    if (lane == 0) pending[w] = c;
}

enum ReqState { kQueued, kRunning, kFinishing, kDone };

// nx, ny, px, py, periodic, sampling stride, subdomain scheme (the schemes use the solver
// vectors differently, so state is reused only within a scheme)
typedef std::tuple<int, int, int, int, int, int, int> ShapeKey;

struct Request {
    int64_t id = 0;
    sdd_params prm{};
    int32_t mon_kind = SDD_MONITOR_NODAL;
    int32_t n_params = 0;
    double mon_params[64] = {0};
    std::vector<double> x0, y0, omega;
    int32_t step_index = 0;
    int M = 0;
    ReqState state = kQueued;
    sdd_status status = SDD_OK;
    sdd_problem* p = nullptr;
    int slot = -1;
    int64_t off = 0;
    int32_t rounds = 0;
    bool cancel = false;            // cancellation asked while running
    cudaEvent_t up_ev = nullptr;    // inputs uploaded (upload stream)
    cudaEvent_t done_ev = nullptr;  // finish work complete (finish stream)
};

ShapeKey shape_of(const sdd_params& q)
{
    return ShapeKey(q.nx, q.ny, q.px, q.py, q.periodic, q.iface_stride > 1 ? q.iface_stride : 1, q.subdomain_scheme);
}

}  // namespace

struct sdd_server {
    sdd_server_params prm{};
    cudaStream_t stream = nullptr;   // rounds: admission kernels, plan, path kernel, reduce
    cudaStream_t up = nullptr;       // host -> device uploads of admitted requests
    cudaStream_t fin = nullptr;      // finishing requests: estimates, scatter, solves
    bool fp64 = false;
    int acc_mode = kAcc64;
    int mc_grid = 1;
    // node pool (device)
    int32_t* node_prob = nullptr;
    double *shift = nullptr, *acc = nullptr, *est = nullptr, *se = nullptr;
    int64_t *n_done = nullptr, *steps = nullptr, *paths_run = nullptr, *next_total = nullptr;
    int64_t *p_begin = nullptr, *p_count = nullptr, *task_off = nullptr;
    int32_t *node_of = nullptr, *n_active = nullptr, *task_counter = nullptr;
    TaskSlot* slots = nullptr;
    int2* slot_range = nullptr;
    int32_t* pending = nullptr;
    int32_t *range_off = nullptr, *range_pre = nullptr;  // planning order of the running ranges
    int32_t* slot_bad = nullptr;     // per slot: invalid monitor or mesh found by the preparation
    void* records = nullptr;         // McProblem<T> per slot (device)
    // pinned host mirrors
    void* h_records = nullptr;
    int2* h_slot_range = nullptr;
    int32_t* h_pending = nullptr;    // [max_resident + 1]: pending per slot, then n_active
    int32_t *h_range_off = nullptr, *h_range_pre = nullptr;
    int32_t* h_bad = nullptr;
    // host bookkeeping
    std::map<int64_t, int64_t> free_ranges;  // offset -> length
    std::vector<int> free_slots;
    std::map<int64_t, Request*> reqs;        // every request not yet collected, by id
    std::deque<Request*> queue;              // QUEUED, arrival order
    std::list<Request*> running;             // RUNNING, admission order
    std::list<Request*> finishing;           // FINISHING
    std::deque<int64_t> done_ids;            // DONE, not yet polled
    std::map<ShapeKey, std::vector<sdd_problem*>> cache;
    std::list<sdd_problem*> cache_order;     // cached problems, oldest first
    int64_t next_id = 1;
    sdd_server_stats st{};
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    bool round_timed = false;
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
            st.pool_bytes += (int64_t)bytes;
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
    ~sdd_server()
    {
        if (stream) cudaStreamSynchronize(stream);
        if (up) cudaStreamSynchronize(up);
        if (fin) cudaStreamSynchronize(fin);
        for (auto& kv : reqs) {
            Request* r = kv.second;
            if (r->up_ev) cudaEventDestroy(r->up_ev);
            if (r->done_ev) cudaEventDestroy(r->done_ev);
            delete r->p;
            delete r;
        }
        for (sdd_problem* p : cache_order) delete p;
        if (ev_a) cudaEventDestroy(ev_a);
        if (ev_b) cudaEventDestroy(ev_b);
        if (up) cudaStreamDestroy(up);
        if (fin) cudaStreamDestroy(fin);
        for (void* v : allocs) cudaFree(v);
        for (void* v : host_allocs) cudaFreeHost(v);
    }
};

namespace {

#define S_CK(call)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            const std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);     \
            return sdd_fail(e_ == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA,  \
                            m_.c_str());                                                   \
        }                                                                                  \
    } while (0)

#define S_TRY(call)                            \
    do {                                       \
        sdd_status s_ = (call);                \
        if (s_ != SDD_OK) return s_;           \
    } while (0)

// First-fit allocation of n contiguous pool nodes; -1 when no range is long enough.
int64_t range_alloc(sdd_server* s, int64_t n)
{
    if (n == 0) return 0;
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second < n) continue;
        const int64_t off = it->first, len = it->second;
        s->free_ranges.erase(it);
        if (len > n) s->free_ranges[off + n] = len - n;
        if (off + n > s->st.pool_high_water) s->st.pool_high_water = off + n;
        return off;
    }
    return -1;
}

void range_free(sdd_server* s, int64_t off, int64_t n)
{
    if (n == 0) return;
    auto it = s->free_ranges.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != s->free_ranges.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_ranges.erase(nx);
    }
    if (it != s->free_ranges.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_ranges.erase(it);
        }
    }
}

bool range_available(const sdd_server* s, int64_t n)
{
    if (n == 0) return true;
    for (const auto& kv : s->free_ranges)
        if (kv.second >= n) return true;
    return false;
}

void evict_oldest(sdd_server* s)
{
    sdd_problem* old = s->cache_order.front();
    s->cache_order.pop_front();
    auto& v = s->cache[shape_of(old->prm)];
    for (size_t k = 0; k < v.size(); ++k)
        if (v[k] == old) {
            v.erase(v.begin() + (long)k);
            break;
        }
    s->st.resident_bytes -= (int64_t)old->dev_bytes;
    s->st.cached_bytes -= (int64_t)old->dev_bytes;
    delete old;  // cudaFree: waits for the device
}

// Device state for a request's shape: a cached one, or a new allocation within the budget
// (evicting cached state of other shapes, oldest first).  *p = nullptr: not now; *never: the
// request cannot fit even with nothing else resident.
sdd_status acquire_problem(sdd_server* s, const Request* r, sdd_problem** p, bool* never)
{
    *p = nullptr;
    *never = false;
    const ShapeKey key = shape_of(r->prm);
    auto it = s->cache.find(key);
    if (it != s->cache.end() && !it->second.empty()) {
        *p = it->second.back();
        it->second.pop_back();
        s->cache_order.remove(*p);
        s->st.cached_bytes -= (int64_t)(*p)->dev_bytes;
        return SDD_OK;
    }
    // requests other than queued ones hold device state
    const bool others_resident = s->reqs.size() > s->queue.size();
    const int64_t need = (int64_t)sdd_problem_device_bytes(r->prm, false);
    const int64_t budget = s->prm.mem_budget_bytes;
    if (budget > 0) {
        if (need > budget) {
            *never = true;
            return SDD_OK;
        }
        while (s->st.resident_bytes + need > budget && !s->cache_order.empty()) evict_oldest(s);
        if (s->st.resident_bytes + need > budget) return SDD_OK;
    }
    for (;;) {
        const sdd_status a = sdd_alloc_problem(r->prm, s->up, false, p);
        if (a == SDD_OK) break;
        if (a != SDD_ERR_OOM) return a;
        *p = nullptr;
        if (!s->cache_order.empty()) {
            evict_oldest(s);  // the device is full: make room from the cache first
            continue;
        }
        *never = !others_resident;  // else wait for resident requests to be collected
        return SDD_OK;
    }
    s->st.resident_bytes += (int64_t)(*p)->dev_bytes;
    s->st.allocations += 1;
    return SDD_OK;
}

void release_problem(sdd_server* s, sdd_problem* p)
{
    s->cache[shape_of(p->prm)].push_back(p);
    s->cache_order.push_back(p);
    s->st.cached_bytes += (int64_t)p->dev_bytes;
}

template <typename T>
void write_record(sdd_server* s, const Request* r)
{
    McProblem<T> R = mc_problem<T>(r->p);
    R.node_offset = (int32_t)r->off;
    static_cast<McProblem<T>*>(s->h_records)[r->slot] = R;
}

// Upload, monitor, estimator shifts and pool-node init of an admitted request.
sdd_status admit(sdd_server* s, Request* r)
{
    sdd_problem* p = r->p;
    p->prm = r->prm;
    p->step = r->step_index;
    p->mon_kind = r->mon_kind;
    p->n_params = r->n_params;
    memcpy(p->mon_params, r->mon_params, sizeof(p->mon_params));
    p->stream = s->stream;
    const size_t N = (size_t)r->prm.nx * r->prm.ny;
    S_CK(cudaMemcpyAsync(p->x, r->x0.data(), N * 8, cudaMemcpyHostToDevice, s->up));
    S_CK(cudaMemcpyAsync(p->y, r->y0.data(), N * 8, cudaMemcpyHostToDevice, s->up));
    if (r->mon_kind == SDD_MONITOR_NODAL)
        S_CK(cudaMemcpyAsync(p->omega_nodal, r->omega.data(), N * 8, cudaMemcpyHostToDevice, s->up));
    S_CK(cudaEventCreateWithFlags(&r->up_ev, cudaEventDisableTiming));
    S_CK(cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming));
    S_CK(cudaEventRecord(r->up_ev, s->up));
    S_CK(cudaStreamWaitEvent(s->stream, r->up_ev, 0));
    PrepParams P{};
    P.nx = r->prm.nx; P.ny = r->prm.ny; P.periodic = r->prm.periodic;
    P.kind = r->mon_kind; P.n_params = r->n_params; P.precision = r->prm.precision;
    P.Lx = r->prm.Lx; P.Ly = r->prm.Ly;
    P.t = r->prm.t0 + (double)r->step_index * r->prm.dt;
    P.x = p->x; P.y = p->y; P.omega_in = p->omega_nodal;
    memcpy(P.params, r->mon_params, sizeof(P.params));
    P.om64 = p->om64; P.wxi64 = p->wxi64; P.weta64 = p->weta64; P.mon = p->mon; P.disp = p->disp;
    P.bad = s->slot_bad + r->slot;
    P.moving_boundary = r->prm.moving_boundary; P.form = r->prm.form; P.r = r->prm.dt / r->prm.tau;
    P.bnd64 = p->bnd64; P.bnd = p->bnd; P.bnd_scratch = p->bnd_scratch;
    S_CK(cudaMemsetAsync(P.bad, 0, 4, s->stream));
    S_CK(launch_prep(P, s->stream));
    s->st.kernel_launches += 2;
    if (r->M > 0) {
        const int64_t o = r->off;
        S_CK(launch_shift(p->nodes, r->M, r->prm.nx, p->x, p->y, s->shift + 2 * o, s->stream));
        fill_i32_kernel<<<(r->M + 255) / 256, 256, 0, s->stream>>>(s->node_prob + o, r->M, r->slot);
        S_CK(cudaGetLastError());
        const bool adaptive = s->prm.se_target > 0;
        const int64_t n0 = s->prm.paths_per_node;
        const int64_t maxp = adaptive ? s->prm.max_paths_per_node : n0;
        S_CK(launch_mc_init(r->M, n0, maxp, s->acc + 4 * o, s->n_done + o, s->steps + o, s->paths_run + o,
                            s->next_total + o, s->stream, p->n_interp > 0 ? p->iface_role : nullptr));
        s->st.kernel_launches += 3;
    }
    if (s->fp64) write_record<double>(s, r); else write_record<float>(s, r);
    const size_t rec = s->fp64 ? sizeof(McProblem<double>) : sizeof(McProblem<float>);
    S_CK(cudaMemcpyAsync(static_cast<char*>(s->records) + rec * r->slot,
                         static_cast<char*>(s->h_records) + rec * r->slot, rec, cudaMemcpyHostToDevice,
                         s->stream));
    s->h_slot_range[r->slot] = int2{(int)r->off, r->M};
    S_CK(cudaMemcpyAsync(s->slot_range + r->slot, s->h_slot_range + r->slot, sizeof(int2),
                         cudaMemcpyHostToDevice, s->stream));
    r->state = kRunning;
    return SDD_OK;
}

// Estimates, Dirichlet scatter and subdomain solves of a request whose nodes are all done.
sdd_status finish(sdd_server* s, Request* r)
{
    sdd_problem* p = r->p;
    const int64_t o = r->off;
    if (r->M > 0) {
        S_CK(launch_output(r->M, s->acc + 4 * o, s->n_done + o, s->shift + 2 * o, s->est + 2 * o, s->se + 2 * o,
                           s->fin));
        S_CK(launch_interp(p->interp, p->n_interp, s->est + 2 * o, s->se + 2 * o, s->fin));
        s->st.kernel_launches += 1 + (p->n_interp > 0 ? 1 : 0);
    }
    S_CK(launch_scatter(r->prm.nx, r->prm.ny, r->prm.periodic, r->prm.Lx, r->prm.Ly, p->nodes, r->M,
                        s->est + 2 * o, p->xn, p->yn, s->fin, r->prm.moving_boundary ? p->bnd64 : nullptr));
    s->st.kernel_launches += (r->prm.periodic ? 0 : 1) + (r->M > 0 ? 1 : 0);
    SolveParams S{};
    S.nx = r->prm.nx; S.ny = r->prm.ny; S.px = r->prm.px; S.py = r->prm.py; S.form = r->prm.form;
    S.r = r->prm.dt / r->prm.tau; S.rtol = r->prm.solve_rtol; S.max_iter = r->prm.solve_max_iter;
    S.scheme = r->prm.subdomain_scheme;
    S.fe_max_substeps = r->prm.fe_max_substeps > 0 ? r->prm.fe_max_substeps : (1 << 16);
    S.om64 = p->om64; S.xcur = p->x; S.ycur = p->y; S.xnew = p->xn; S.ynew = p->yn;
    S.ce64 = p->ce64; S.cn64 = p->cn64; S.ce = p->ce; S.cn = p->cn; S.vec = p->vec;
    S.mg = p->mg; S.mg_stride = p->mg_stride;
    S.stat_iters = p->st_iters; S.stat_outer = p->st_outer; S.stat_ok = p->st_ok; S.stat_res = p->st_res;
    if (!p->h_items.empty())
        S_CK(launch_solve_items(S, p->solve_items, (int)p->h_items.size(), s->fp64, s->fin));
    else
        S_CK(launch_solve(S, s->fp64, s->fin));
    s->st.kernel_launches += 2;
    S_CK(cudaEventRecord(r->done_ev, s->fin));
    r->state = kFinishing;
    return SDD_OK;
}

template <typename T>
sdd_status launch_round(sdd_server* s, int hw)
{
    McParams<T> P{};
    P.probs = static_cast<const McProblem<T>*>(s->records);
    P.node_prob = s->node_prob;
    P.shift = s->shift;
    P.node_of = s->node_of; P.p_begin = s->p_begin; P.p_count = s->p_count; P.task_off = s->task_off;
    P.n_active = s->n_active; P.task_counter = s->task_counter; P.slots = s->slots;
    // the problem switches, when every running request shares them (the path kernel then has
    // them compiled in; each request's results are the same either way)
    int mode = -1;
    bool first = true;
    for (const Request* r : s->running) {
        const int m = (r->prm.periodic ? 1 : 0) | (r->prm.form ? 2 : 0) | (r->prm.bb_test ? 4 : 0);
        mode = first ? m : (mode == m ? m : -1);
        first = false;
    }
    S_CK(cudaEventRecord(s->ev_a, s->stream));
    S_CK(launch_mc<T>(P, s->acc_mode, false, true, s->mc_grid, s->stream, 256, mode));
    S_CK(cudaEventRecord(s->ev_b, s->stream));
    ReduceParams RP{};
    RP.node_of = s->node_of; RP.p_count = s->p_count; RP.task_off = s->task_off; RP.n_active = s->n_active;
    RP.slots = s->slots; RP.shift = s->shift; RP.acc = s->acc; RP.n_done = s->n_done; RP.steps = s->steps;
    RP.paths_run = s->paths_run; RP.next_total = s->next_total;
    const bool adaptive = s->prm.se_target > 0;
    RP.se_target = adaptive ? s->prm.se_target : 0.0;
    RP.max_paths = adaptive ? s->prm.max_paths_per_node : s->prm.paths_per_node;
    S_CK(launch_reduce(RP, hw, s->stream));
    s->st.kernel_launches += 2;
    s->st.rounds += 1;
    s->round_timed = true;
    return SDD_OK;
}

void count_states(const sdd_server* s, sdd_server_stats* o)
{
    o->queued = (int32_t)s->queue.size();
    o->running = (int32_t)s->running.size();
    o->finishing = (int32_t)s->finishing.size();
    int32_t done = 0;
    for (const auto& kv : s->reqs) done += kv.second->state == kDone ? 1 : 0;
    o->done = done;
}

void complete(sdd_server* s, Request* r)
{
    r->state = kDone;
    s->done_ids.push_back(r->id);
    s->st.completed += 1;
    if (r->status == SDD_OK) s->st.interface_nodes += r->M;
}

}  // namespace

extern "C" {

sdd_status sdd_server_create(const sdd_server_params* params, void* stream, sdd_server** out)
{
    if (!out) return sdd_fail(SDD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!params) return sdd_fail(SDD_ERR_INVALID_ARG, "params is NULL");
    const sdd_server_params& q = *params;
    if (!stream) return sdd_fail(SDD_ERR_INVALID_ARG, "the server needs a non-NULL stream");
    if (q.precision < SDD_FP64 || q.precision > SDD_FP32_KAHAN) return sdd_fail(SDD_ERR_INVALID_ARG, "bad precision");
    if (q.max_resident < 1 || q.max_resident > (1 << 16))
        return sdd_fail(SDD_ERR_INVALID_ARG, "max_resident must be in [1, 2^16]");
    if (q.max_nodes < 1 || q.max_nodes >= ((int64_t)1 << 23))  // a round's tasks fit in an int
        return sdd_fail(SDD_ERR_INVALID_ARG, "max_nodes must be in [1, 2^23)");
    if (q.mem_budget_bytes < 0) return sdd_fail(SDD_ERR_INVALID_ARG, "mem_budget_bytes must be >= 0");
    if (q.round_paths < 0) return sdd_fail(SDD_ERR_INVALID_ARG, "round_paths must be >= 0");
    if (!(q.se_target >= 0) || !isfinite(q.se_target)) return sdd_fail(SDD_ERR_INVALID_ARG, "se_target must be >= 0");
    if (q.paths_per_node < 2) return sdd_fail(SDD_ERR_INVALID_ARG, "paths_per_node must be >= 2");
    const int64_t cap = q.se_target > 0 ? q.max_paths_per_node : q.paths_per_node;
    if (cap < q.paths_per_node || cap > ((int64_t)1 << 31))
        return sdd_fail(SDD_ERR_INVALID_ARG, "max_paths_per_node must be in [paths_per_node, 2^31]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return sdd_fail(SDD_ERR_NO_DEVICE, "no CUDA device visible");
    }
    sdd_server* s = new sdd_server();
    s->prm = q;
    s->stream = static_cast<cudaStream_t>(stream);
    s->fp64 = q.precision == SDD_FP64;
    s->acc_mode = q.precision == SDD_FP32_KAHAN ? kAccKahan32 : kAcc64;
    const size_t M = (size_t)q.max_nodes + 1;
    const size_t R = (size_t)q.max_resident;
    const size_t rec = s->fp64 ? sizeof(McProblem<double>) : sizeof(McProblem<float>);
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) if (e == cudaSuccess) e = s->dalloc(&(ptr), (bytes))
#define HALLOC(ptr, bytes) if (e == cudaSuccess) e = s->halloc(&(ptr), (bytes))
    ALLOC(s->node_prob, M * 4); ALLOC(s->shift, M * 16); ALLOC(s->acc, M * 32); ALLOC(s->est, M * 16);
    ALLOC(s->se, M * 16); ALLOC(s->n_done, M * 8); ALLOC(s->steps, M * 8); ALLOC(s->paths_run, M * 8);
    ALLOC(s->next_total, M * 8); ALLOC(s->p_begin, M * 8); ALLOC(s->p_count, M * 8);
    ALLOC(s->task_off, (M + 1) * 8); ALLOC(s->node_of, M * 4); ALLOC(s->n_active, 16);
    ALLOC(s->task_counter, 16); ALLOC(s->slots, M * kSlotsPerNode * sizeof(TaskSlot));
    ALLOC(s->slot_range, R * sizeof(int2)); ALLOC(s->pending, (R + 1) * 4); ALLOC(s->records, rec * R);
    ALLOC(s->range_off, (R + 1) * 4); ALLOC(s->range_pre, (R + 1) * 4); ALLOC(s->slot_bad, R * 4);
    HALLOC(s->h_records, rec * R); HALLOC(s->h_slot_range, R * sizeof(int2)); HALLOC(s->h_pending, (R + 2) * 4);
    HALLOC(s->h_range_off, (R + 1) * 4); HALLOC(s->h_range_pre, (R + 1) * 4); HALLOC(s->h_bad, R * 4);
#undef ALLOC
#undef HALLOC
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->fin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_b);
    // idle pool nodes are never scheduled: n_done = next_total = 0; empty slot ranges
    if (e == cudaSuccess) e = cudaMemsetAsync(s->n_done, 0, M * 8, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->next_total, 0, M * 8, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->slot_range, 0, R * sizeof(int2), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const std::string m = std::string("server allocation failed: ") + cudaGetErrorString(e);
        delete s;
        return sdd_fail(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, m.c_str());
    }
    memset(s->h_slot_range, 0, R * sizeof(int2));
    s->free_ranges[0] = q.max_nodes;
    for (int k = (int)R - 1; k >= 0; --k) s->free_slots.push_back(k);
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    s->mc_grid = nsm * (s->fp64 ? mc_max_blocks_per_sm<double>(s->acc_mode, false, true)
                                : mc_max_blocks_per_sm<float>(s->acc_mode, false, true));
    *out = s;
    return SDD_OK;
}

sdd_status sdd_server_submit(sdd_server* s, const sdd_params* params, const double* x0, const double* y0,
                             int32_t monitor_kind, const double* monitor_params, int32_t n_params,
                             const double* omega, int32_t step_index, int64_t* id)
{
    if (!s || !id) return sdd_fail(SDD_ERR_INVALID_ARG, "NULL argument");
    *id = 0;
    S_TRY(sdd_validate_params(params));
    const sdd_params& q = *params;
    const sdd_server_params& v = s->prm;
    if (q.precision != v.precision || q.se_target != v.se_target || q.paths_per_node != v.paths_per_node ||
        (v.se_target > 0 && q.max_paths_per_node != v.max_paths_per_node))
        return sdd_fail(SDD_ERR_INVALID_ARG, "precision, se_target and path counts must equal the server's");
    if (!x0 || !y0) return sdd_fail(SDD_ERR_INVALID_ARG, "x0, y0 must not be NULL");
    if (step_index < 0) return sdd_fail(SDD_ERR_INVALID_ARG, "step_index must be >= 0");
    if (monitor_kind == SDD_MONITOR_GAUSS && n_params != 4) return sdd_fail(SDD_ERR_INVALID_ARG, "GAUSS needs 4 params");
    if (monitor_kind == SDD_MONITOR_FRONT && n_params != 6) return sdd_fail(SDD_ERR_INVALID_ARG, "FRONT needs 6 params");
    if (monitor_kind == SDD_MONITOR_BUMPS && (n_params % 4 || n_params < 0 || n_params > 64))
        return sdd_fail(SDD_ERR_INVALID_ARG, "BUMPS needs 4k params, k <= 16");
    if (monitor_kind == SDD_MONITOR_RINGS && (n_params < 5 || (n_params - 3) % 2 || n_params > 63))
        return sdd_fail(SDD_ERR_INVALID_ARG, "RINGS needs 3 + 2k params, 1 <= k <= 30");
    if (monitor_kind < SDD_MONITOR_NODAL || monitor_kind > SDD_MONITOR_RINGS)
        return sdd_fail(SDD_ERR_INVALID_ARG, "bad monitor kind");
    if (monitor_kind == SDD_MONITOR_NODAL && n_params != 0)
        return sdd_fail(SDD_ERR_INVALID_ARG, "NODAL takes omega, not params");
    if (n_params > 0 && !monitor_params) return sdd_fail(SDD_ERR_INVALID_ARG, "monitor_params is NULL");
    std::vector<int32_t> ij;
    sdd_layout(q.nx, q.ny, q.px, q.py, q.periodic, ij);
    const int M = (int)(ij.size() / 2);
    if (M > v.max_nodes) return sdd_fail(SDD_ERR_INVALID_ARG, "request has more interface nodes than the pool");
    if (!sdd_boundary_ok(q, x0, y0))
        return sdd_fail(SDD_ERR_INVALID_ARG, "Dirichlet mesh must equal (Lx xi, Ly eta) on the boundary");
    const size_t N = (size_t)q.nx * q.ny;
    Request* r = new Request();
    r->id = s->next_id++;
    r->prm = q;
    r->mon_kind = monitor_kind;
    r->n_params = n_params;
    for (int k = 0; k < n_params; ++k) r->mon_params[k] = monitor_params[k];
    r->x0.assign(x0, x0 + N);
    r->y0.assign(y0, y0 + N);
    if (monitor_kind == SDD_MONITOR_NODAL) {
        if (omega) r->omega.assign(omega, omega + N);
        else r->omega.assign(N, 1.0);
    }
    r->step_index = step_index;
    r->M = M;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    s->st.submitted += 1;
    *id = r->id;
    return SDD_OK;
}

sdd_status sdd_server_progress(sdd_server* s, int32_t* n_running, int32_t* n_queued)
{
    if (!s) return sdd_fail(SDD_ERR_INVALID_ARG, "server is NULL");
    const TraceRange trace("sdd_server_progress");
    // 1. finishing requests whose work is complete
    for (auto it = s->finishing.begin(); it != s->finishing.end();) {
        Request* r = *it;
        const cudaError_t q = cudaEventQuery(r->done_ev);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        S_CK(q);
        complete(s, r);
        it = s->finishing.erase(it);
    }
    // 2. admission, first come first served
    while (!s->queue.empty()) {
        Request* r = s->queue.front();
        if (s->free_slots.empty() || !range_available(s, r->M)) break;
        sdd_problem* p = nullptr;
        bool never = false;
        S_TRY(acquire_problem(s, r, &p, &never));
        if (never) {
            s->queue.pop_front();
            r->status = SDD_ERR_OOM;
            complete(s, r);
            continue;
        }
        if (!p) break;
        s->queue.pop_front();
        r->p = p;
        r->slot = s->free_slots.back();
        s->free_slots.pop_back();
        r->off = range_alloc(s, r->M);
        S_TRY(admit(s, r));
        s->running.push_back(r);
    }
    // 3. plan the running requests' nodes, oldest request first; pending nodes per slot
    if (!s->running.empty()) {
        int hw = 0, nr = 0;
        for (const Request* r : s->running) {
            if (r->M == 0) continue;
            s->h_range_off[nr] = (int32_t)r->off;
            s->h_range_pre[nr] = hw;
            hw += r->M;
            ++nr;
        }
        s->h_range_pre[nr] = hw;
        const int R = s->prm.max_resident;
        if (hw > 0) {
            S_CK(cudaMemcpyAsync(s->range_off, s->h_range_off, (size_t)nr * 4, cudaMemcpyHostToDevice, s->stream));
            S_CK(cudaMemcpyAsync(s->range_pre, s->h_range_pre, (size_t)(nr + 1) * 4, cudaMemcpyHostToDevice,
                                 s->stream));
            PlanParams PP{};
            PP.M = hw; PP.n_done = s->n_done; PP.next_total = s->next_total; PP.node_of = s->node_of;
            PP.p_begin = s->p_begin; PP.p_count = s->p_count; PP.task_off = s->task_off;
            PP.n_active = s->n_active; PP.task_counter = s->task_counter;
            PP.range_off = s->range_off; PP.range_pre = s->range_pre; PP.n_ranges = nr;
            PP.max_tasks = (s->prm.round_paths + kPathsPerTask - 1) / kPathsPerTask;
            S_CK(launch_plan(PP, s->stream));
            slot_pending_kernel<<<(R * 32 + 255) / 256, 256, 0, s->stream>>>(s->slot_range, R, s->n_done,
                                                                              s->next_total, s->pending);
            S_CK(cudaGetLastError());
            S_CK(cudaMemcpyAsync(s->h_pending, s->pending, (size_t)R * 4, cudaMemcpyDeviceToHost, s->stream));
            S_CK(cudaMemcpyAsync(s->h_pending + R, s->n_active, 4, cudaMemcpyDeviceToHost, s->stream));
            s->st.kernel_launches += 2;
        }
        S_CK(cudaMemcpyAsync(s->h_bad, s->slot_bad, (size_t)R * 4, cudaMemcpyDeviceToHost, s->stream));
        S_CK(cudaStreamSynchronize(s->stream));
        if (s->round_timed) {
            float ms = 0.f;
            S_CK(cudaEventElapsedTime(&ms, s->ev_a, s->ev_b));
            s->st.mc_kernel_ms += ms;
            s->round_timed = false;
        }
        const int n_active = hw > 0 ? s->h_pending[R] : 0;
        // 4. finish requests whose nodes are all done; drop requests with invalid input (their
        //    nodes leave the plan; a round already launched may still sample them)
        for (auto it = s->running.begin(); it != s->running.end();) {
            Request* r = *it;
            if (s->h_bad[r->slot] || r->cancel) {
                r->status = r->cancel ? SDD_ERR_CANCELLED : SDD_ERR_INVALID_ARG;
                complete(s, r);
                it = s->running.erase(it);
                continue;
            }
            if (r->M > 0 && s->h_pending[r->slot] > 0) {
                r->rounds += 1;
                ++it;
                continue;
            }
            S_TRY(finish(s, r));
            s->finishing.push_back(r);
            it = s->running.erase(it);
        }
        // 5. the next round over every running request's pending nodes
        if (n_active > 0) {
            if (s->fp64) S_TRY(launch_round<double>(s, hw));
            else S_TRY(launch_round<float>(s, hw));
        }
    }
    if (n_running) *n_running = (int32_t)s->running.size();
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    return SDD_OK;
}

sdd_status sdd_server_poll(sdd_server* s, int64_t* ids, int32_t cap, int32_t* n)
{
    if (!s || !n || cap < 0 || (cap > 0 && !ids)) return sdd_fail(SDD_ERR_INVALID_ARG, "bad arguments");
    int32_t k = 0;
    while (k < cap && !s->done_ids.empty()) {
        ids[k++] = s->done_ids.front();
        s->done_ids.pop_front();
    }
    *n = k;
    return SDD_OK;
}

sdd_status sdd_server_result(sdd_server* s, int64_t id, double* x, double* y, double* est_xy, double* se_xy,
                             sdd_stats* st)
{
    if (!s) return sdd_fail(SDD_ERR_INVALID_ARG, "server is NULL");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sdd_fail(SDD_ERR_INVALID_ARG, "unknown request id");
    Request* r = it->second;
    if (r->state != kDone) return sdd_fail(SDD_ERR_INVALID_ARG, "request not completed");
    sdd_status status = r->status;
    if (r->p && (status == SDD_ERR_INVALID_ARG || status == SDD_ERR_CANCELLED)) {
        if (st) *st = sdd_stats{};
    } else if (r->p) {
        sdd_problem* p = r->p;
        const size_t N = (size_t)r->prm.nx * r->prm.ny;
        const int64_t o = r->off;
        const int M = r->M;
        if (x) S_CK(cudaMemcpyAsync(x, p->xn, N * 8, cudaMemcpyDefault, s->fin));
        if (y) S_CK(cudaMemcpyAsync(y, p->yn, N * 8, cudaMemcpyDefault, s->fin));
        if (est_xy && M > 0) S_CK(cudaMemcpyAsync(est_xy, s->est + 2 * o, (size_t)M * 16, cudaMemcpyDefault, s->fin));
        if (se_xy && M > 0) S_CK(cudaMemcpyAsync(se_xy, s->se + 2 * o, (size_t)M * 16, cudaMemcpyDefault, s->fin));
        const int ns = r->prm.px * r->prm.py;
        std::vector<int64_t> stp((size_t)M + 1), npr((size_t)M + 1);
        std::vector<double> sev((size_t)2 * M + 2);
        std::vector<int32_t> it_(ns), ou(ns), ok(ns);
        std::vector<double> rs(ns);
        if (M > 0) {
            S_CK(cudaMemcpyAsync(stp.data(), s->steps + o, (size_t)M * 8, cudaMemcpyDeviceToHost, s->fin));
            S_CK(cudaMemcpyAsync(npr.data(), s->paths_run + o, (size_t)M * 8, cudaMemcpyDeviceToHost, s->fin));
            S_CK(cudaMemcpyAsync(sev.data(), s->se + 2 * o, (size_t)M * 16, cudaMemcpyDeviceToHost, s->fin));
        }
        S_CK(cudaMemcpyAsync(it_.data(), p->st_iters, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s->fin));
        S_CK(cudaMemcpyAsync(ou.data(), p->st_outer, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s->fin));
        S_CK(cudaMemcpyAsync(ok.data(), p->st_ok, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s->fin));
        S_CK(cudaMemcpyAsync(rs.data(), p->st_res, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s->fin));
        S_CK(cudaStreamSynchronize(s->fin));
        sdd_stats o_{};
        o_.M = M;
        o_.step_index = r->step_index + 1;
        o_.t = r->prm.t0 + (double)(r->step_index + 1) * r->prm.dt;
        o_.mc_rounds = r->rounds;
        int bad = 0;
        for (int m = 0; m < M; ++m) {
            o_.path_steps += stp[m];
            o_.paths += npr[m];
            const double v = sev[2 * m] > sev[2 * m + 1] ? sev[2 * m] : sev[2 * m + 1];
            if (v > o_.max_se) o_.max_se = v;
            if (s->prm.se_target > 0 && v > s->prm.se_target) o_.nodes_not_reached += 1;
        }
        for (int k = 0; k < ns; ++k) {
            if (it_[k] > o_.solve_iters_max) o_.solve_iters_max = it_[k];
            if (ou[k] > o_.solve_outer_max) o_.solve_outer_max = ou[k];
            if (rs[k] > o_.solve_rel_residual) o_.solve_rel_residual = rs[k];
            bad += ok[k] ? 0 : 1;
        }
        s->st.path_steps += o_.path_steps;
        if (st) *st = o_;
        if (o_.nodes_not_reached) status = SDD_ERR_SE_NOT_REACHED;
        else if (bad) status = SDD_ERR_NOT_CONVERGED;
    } else if (st) {
        *st = sdd_stats{};
    }
    if (r->p) {
        sdd_problem* p = r->p;
        // release: state to the shape cache, pool range, slot
        s->h_slot_range[r->slot] = int2{0, 0};
        S_CK(cudaMemcpyAsync(s->slot_range + r->slot, s->h_slot_range + r->slot, sizeof(int2),
                             cudaMemcpyHostToDevice, s->stream));
        range_free(s, r->off, r->M);
        s->free_slots.push_back(r->slot);
        release_problem(s, p);
        r->p = nullptr;
    }
    if (r->up_ev) cudaEventDestroy(r->up_ev);
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    s->reqs.erase(it);
    delete r;
    s->st.collected += 1;
    if (status == SDD_ERR_OOM) return sdd_fail(SDD_ERR_OOM, "request state does not fit the memory budget");
    if (status == SDD_ERR_INVALID_ARG) return sdd_fail(status, "monitor must be finite and > 0, mesh finite");
    if (status == SDD_ERR_CANCELLED) return sdd_fail(status, "request cancelled");
    if (status == SDD_ERR_SE_NOT_REACHED) return sdd_fail(status, "max_paths_per_node reached before se_target");
    if (status == SDD_ERR_NOT_CONVERGED) return sdd_fail(status, "a subdomain solve reached solve_max_iter");
    return status;
}

sdd_status sdd_server_cancel(sdd_server* s, int64_t id)
{
    if (!s) return sdd_fail(SDD_ERR_INVALID_ARG, "server is NULL");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sdd_fail(SDD_ERR_INVALID_ARG, "unknown request id");
    Request* r = it->second;
    if (r->state == kQueued) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == r) {
                s->queue.erase(q);
                break;
            }
        r->status = SDD_ERR_CANCELLED;
        complete(s, r);
    } else if (r->state == kRunning) {
        r->cancel = true;
    }
    return SDD_OK;
}

sdd_status sdd_server_get_stats(sdd_server* s, sdd_server_stats* out)
{
    if (!s || !out) return sdd_fail(SDD_ERR_INVALID_ARG, "NULL argument");
    *out = s->st;
    count_states(s, out);
    return SDD_OK;
}

void sdd_server_destroy(sdd_server* s)
{
    delete s;
}

}  // extern "C"
