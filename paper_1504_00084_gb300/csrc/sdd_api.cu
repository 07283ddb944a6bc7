// C ABI of the SDD mesh generator (declared in include/sdd.h).
//
// Host-side orchestration only: validation, device state, the round loop of the interface
// Monte Carlo, and the order of the kernels of one alternating step.  Every arithmetic step
// of the method runs in the kernels of sdd_prep.cu, sdd_mc.cu and sdd_solve.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <algorithm>
#include <vector>

#include "sdd.h"
#include "sdd_internal.cuh"
#include "sdd_problem.cuh"

using namespace sdd;

namespace {

thread_local std::string g_err;

sdd_status fail(sdd_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

}  // namespace

sdd_status sdd_fail(sdd_status s, const char* msg) { return fail(s, msg); }

namespace {

#define SDD_CK(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

#define SDD_TRY(call)                          \
    do {                                       \
        sdd_status s_ = (call);                \
        if (s_ != SDD_OK) return s_;           \
    } while (0)

constexpr int kSlotsPerNode = kTasksPerRound;  // task slots per node: one round's tasks
constexpr int64_t kMaxNodes = int64_t(1) << 23;  // kMaxNodes * kSlotsPerNode tasks fit in an int
constexpr int kMaxAdaptiveRounds = 4096;
const char kCkptMagic[8] = {'S', 'D', 'D', 'C', 'K', 'P', 'T', '1'};

void layout(int nx, int ny, int px, int py, int periodic, std::vector<int32_t>& ij)
{
    ij.clear();
    std::vector<int> vl, hl;
    for (int I = periodic ? 0 : 1; I < px; ++I) vl.push_back(split_line(I, nx, px));
    for (int J = periodic ? 0 : 1; J < py; ++J) hl.push_back(split_line(J, ny, py));
    const int jlo = periodic ? 0 : 1, jhi = periodic ? ny - 2 : ny - 2;
    const int ilo = periodic ? 0 : 1, ihi = periodic ? nx - 2 : nx - 2;
    std::vector<char> on_v(nx, 0);
    for (int i : vl) on_v[i] = 1;
    for (int i : vl)
        for (int j = jlo; j <= jhi; ++j) { ij.push_back(i); ij.push_back(j); }
    for (int j : hl)
        for (int i = ilo; i <= ihi; ++i)
            if (!on_v[i]) { ij.push_back(i); ij.push_back(j); }
}

// Interface sampling (Sec. 3.6): along every interface line the nodes whose index along the line
// is a multiple of k, and the crossings with lines of the other direction, are estimated; every
// other node is the linear interpolation, in its index along the line, between the nearest
// sampled positions on either side, where a line's end stands for a sample: the identity
// boundary node on a Dirichlet domain, the line's first node one period on when periodic.
void sampling_table(const sdd_params& q, const std::vector<int32_t>& ij, std::vector<int32_t>& role,
                    std::vector<InterpRule>& rules)
{
    const int M = (int)(ij.size() / 2);
    role.assign(M, -1);
    rules.clear();
    const int k = q.iface_stride;
    if (k <= 1 || M == 0) return;
    const int nx = q.nx, ny = q.ny;
    std::vector<int32_t> id((size_t)nx * ny, -1);
    for (int m = 0; m < M; ++m) id[(size_t)ij[2 * m + 1] * nx + ij[2 * m]] = m;
    std::vector<char> is_vl(nx, 0), is_hl(ny, 0);
    std::vector<int> vl, hl;
    for (int I = q.periodic ? 0 : 1; I < q.px; ++I) {
        vl.push_back(split_line(I, nx, q.px));
        is_vl[vl.back()] = 1;
    }
    for (int J = q.periodic ? 0 : 1; J < q.py; ++J) {
        hl.push_back(split_line(J, ny, q.py));
        is_hl[hl.back()] = 1;
    }
    struct Anchor { int t; int32_t node; double ox, oy; };
    auto line = [&](bool vertical, int c) {
        const int L = vertical ? ny - 1 : nx - 1;
        std::vector<Anchor> an;
        for (int t = 0; t <= L; ++t) {
            const int i = vertical ? c : t, j = vertical ? t : c;
            const bool end = t == 0 || t == L;
            if (end && !q.periodic) {
                an.push_back({t, -1, q.Lx * ((double)i / (double)(nx - 1)), q.Ly * ((double)j / (double)(ny - 1))});
            } else if (end && t == L) {
                const int32_t first = vertical ? id[(size_t)c] : id[(size_t)c * nx];
                an.push_back({t, first, vertical ? 0.0 : q.Lx, vertical ? q.Ly : 0.0});
            } else if (t % k == 0 || (vertical ? is_hl[j] : is_vl[i])) {
                an.push_back({t, id[(size_t)j * nx + i], 0.0, 0.0});
            }
        }
        size_t a = 0;
        for (int t = 1; t < L; ++t) {
            while (a + 1 < an.size() && an[a + 1].t <= t) ++a;
            if (an[a].t == t) continue;  // sampled
            const int i = vertical ? c : t, j = vertical ? t : c;
            const int32_t m = id[(size_t)j * nx + i];
            if (m < 0) continue;
            const Anchor& A0 = an[a];
            const Anchor& B0 = an[a + 1];
            InterpRule r{};
            r.m = m;
            r.a = A0.node;
            r.b = B0.node;
            r.w = (double)(B0.t - t) / (double)(B0.t - A0.t);
            r.oax = A0.ox; r.oay = A0.oy; r.obx = B0.ox; r.oby = B0.oy;
            role[m] = (int32_t)rules.size();
            rules.push_back(r);
        }
    };
    for (int i : vl) line(true, i);
    for (int j : hl) line(false, j);
}

bool is_device_ptr(const void* ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace {

sdd_status validate(const sdd_params* P)
{
    if (!P) return fail(SDD_ERR_INVALID_ARG, "params is NULL");
    if (P->nx < 3 || P->ny < 3) return fail(SDD_ERR_INVALID_ARG, "nx, ny must be >= 3");
    if ((int64_t)P->nx * P->ny > (int64_t)1 << 28) return fail(SDD_ERR_INVALID_ARG, "grid too large");
    if (P->px < 1 || P->py < 1) return fail(SDD_ERR_INVALID_ARG, "px, py must be >= 1");
    if (P->px > P->nx - 1 || P->py > P->ny - 1)
        return fail(SDD_ERR_INVALID_ARG, "px <= nx - 1 and py <= ny - 1 (every subdomain spans a cell)");
    {
        // interface nodes in closed form; a round's tasks (up to kSlotsPerNode per node) are
        // counted in 32 bits
        const int64_t nx = P->nx, ny = P->ny, px = P->px, py = P->py;
        const int64_t M = P->periodic ? px * (ny - 1) + py * (nx - 1) - px * py
                                      : (px - 1) * (ny - 2) + (py - 1) * (nx - 2) - (px - 1) * (py - 1);
        if (M >= kMaxNodes) return fail(SDD_ERR_INVALID_ARG, "interface nodes must number below 2^23");
    }
    if (P->periodic != 0 && P->periodic != 1) return fail(SDD_ERR_INVALID_ARG, "periodic must be 0 or 1");
    if (P->form != SDD_FORM_DIV && P->form != SDD_FORM_WINSLOW) return fail(SDD_ERR_INVALID_ARG, "bad form");
    if (P->precision < SDD_FP64 || P->precision > SDD_FP32_KAHAN)
        return fail(SDD_ERR_INVALID_ARG, "bad precision");
    if (P->bicubic != 0 && P->bicubic != 1) return fail(SDD_ERR_INVALID_ARG, "bicubic must be 0 or 1");
    if (P->bb_test != 0 && P->bb_test != 1) return fail(SDD_ERR_INVALID_ARG, "bb_test must be 0 or 1");
    if (P->substeps < 1 || P->substeps > (1 << 20)) return fail(SDD_ERR_INVALID_ARG, "substeps must be in [1, 2^20]");
    if (P->solve_max_iter < 1) return fail(SDD_ERR_INVALID_ARG, "solve_max_iter must be >= 1");
    if (P->iface_stride < 0 || P->iface_stride > (1 << 16)) return fail(SDD_ERR_INVALID_ARG, "iface_stride must be in [0, 2^16]");
    if (!(P->Lx > 0) || !(P->Ly > 0) || !(P->tau > 0) || !(P->dt > 0))
        return fail(SDD_ERR_INVALID_ARG, "Lx, Ly, tau, dt must be > 0");
    if (!isfinite(P->Lx) || !isfinite(P->Ly) || !isfinite(P->tau) || !isfinite(P->dt) || !isfinite(P->t0))
        return fail(SDD_ERR_INVALID_ARG, "non-finite parameter");
    if (P->paths_per_node < 2) return fail(SDD_ERR_INVALID_ARG, "paths_per_node must be >= 2");
    if (!(P->se_target >= 0) || !isfinite(P->se_target)) return fail(SDD_ERR_INVALID_ARG, "se_target must be >= 0");
    const int64_t cap = P->se_target > 0 ? P->max_paths_per_node : P->paths_per_node;
    if (cap < P->paths_per_node || cap > ((int64_t)1 << 31))
        return fail(SDD_ERR_INVALID_ARG, "max_paths_per_node must be in [paths_per_node, 2^31]");
    if (!(P->solve_rtol > 0)) return fail(SDD_ERR_INVALID_ARG, "solve_rtol must be > 0");
    if (P->subdomain_scheme != 0 && P->subdomain_scheme != 1)
        return fail(SDD_ERR_INVALID_ARG, "subdomain_scheme must be 0 or 1");
    if (P->fe_max_substeps < 0) return fail(SDD_ERR_INVALID_ARG, "fe_max_substeps must be >= 0");
    if (P->moving_boundary != 0 && P->moving_boundary != 1)
        return fail(SDD_ERR_INVALID_ARG, "moving_boundary must be 0 or 1");
    if (P->moving_boundary && P->periodic) return fail(SDD_ERR_INVALID_ARG, "a periodic domain has no boundary to move");
    return SDD_OK;
}

sdd_status copy_in(sdd_problem* p, void* dst, const void* src, size_t bytes)
{
    SDD_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, p->stream));
    return SDD_OK;
}

// Copy to a caller buffer; return only after a host destination holds the data.
sdd_status copy_out(sdd_problem* p, void* dst, const void* src, size_t bytes)
{
    if (!dst || bytes == 0) return SDD_OK;
    SDD_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, p->stream));
    if (!is_device_ptr(dst)) SDD_CK(cudaStreamSynchronize(p->stream));
    return SDD_OK;
}

sdd_status check_boundary(const sdd_problem* p, const double* x, const double* y)
{
    if (p->prm.periodic) return SDD_OK;
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    std::vector<double> hx(N), hy(N);
    if (cudaMemcpy(hx.data(), x, N * 8, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(hy.data(), y, N * 8, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(SDD_ERR_INVALID_ARG, "mesh pointers are not readable");
    }
    if (!sdd_boundary_ok(p->prm, hx.data(), hy.data()))
        return fail(SDD_ERR_INVALID_ARG, p->prm.moving_boundary
                                             ? "boundary mesh must have x = 0, Lx on xi = 0, 1 and y = 0, Ly on eta = 0, 1"
                                             : "Dirichlet mesh must equal (Lx xi, Ly eta) on the boundary");
    return SDD_OK;
}

// Monitor on the current mesh, FD gradient, packed records, estimator shifts.
sdd_status run_prep(sdd_problem* p)
{
    const TraceRange trace("sdd: monitor preparation");
    PrepParams P{};
    P.nx = p->prm.nx; P.ny = p->prm.ny; P.periodic = p->prm.periodic;
    P.kind = p->mon_kind; P.n_params = p->n_params; P.precision = p->prm.precision;
    P.Lx = p->prm.Lx; P.Ly = p->prm.Ly;
    P.t = p->monitor_time_fixed ? p->t_monitor : p->prm.t0 + (double)p->step * p->prm.dt;
    P.x = p->x; P.y = p->y; P.omega_in = p->omega_nodal;
    memcpy(P.params, p->mon_params, sizeof(P.params));
    P.om64 = p->om64; P.wxi64 = p->wxi64; P.weta64 = p->weta64;
    P.mon = p->mon; P.disp = p->disp; P.bad = p->bad;
    P.moving_boundary = p->prm.moving_boundary; P.form = p->prm.form; P.r = p->prm.dt / p->prm.tau;
    P.bnd64 = p->bnd64; P.bnd = p->bnd; P.bnd_scratch = p->bnd_scratch;
    SDD_CK(cudaMemsetAsync(p->bad, 0, 4, p->stream));
    SDD_CK(launch_prep(P, p->stream));
    p->launches += 2;
    if (p->M > 0) {
        SDD_CK(launch_shift(p->nodes, p->M, p->prm.nx, p->x, p->y, p->shift, p->stream));
        p->launches += 1;
    }
    return SDD_OK;
}

template <typename T>
McParams<T> mc_params(const sdd_problem* p)
{
    McParams<T> P{};
    P.prob = mc_problem<T>(p);
    P.shift = p->shift;
    P.node_of = p->node_of; P.p_begin = p->p_begin; P.p_count = p->p_count;
    P.task_off = p->task_off; P.n_active = p->n_active; P.task_counter = p->task_counter;
    P.slots = p->slots;
    P.task_paths = p->task_paths;
    return P;
}

sdd_status launch_mc_round(sdd_problem* p, bool debug, double* dval, int32_t* dsteps, int8_t* dside,
                           int64_t dp0, int64_t dn)
{
    if (p->fp64) {
        McParams<double> P = mc_params<double>(p);
        P.dbg_val = dval; P.dbg_steps = dsteps; P.dbg_side = dside; P.dbg_p0 = dp0; P.dbg_n = dn;
        SDD_CK(launch_mc<double>(P, p->acc_mode, debug, false, p->mc_grid, p->stream));
    } else {
        McParams<float> P = mc_params<float>(p);
        P.dbg_val = dval; P.dbg_steps = dsteps; P.dbg_side = dside; P.dbg_p0 = dp0; P.dbg_n = dn;
        SDD_CK(launch_mc<float>(P, p->acc_mode, debug, false, p->mc_grid, p->stream));
    }
    return SDD_OK;
}

// Path-kernel launch bracketed by CUDA events on the problem's stream (pair `slot`).
sdd_status timed_mc_round(sdd_problem* p, int slot)
{
    while ((int)p->ev.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        SDD_CK(cudaEventCreate(&e));
        p->ev.push_back(e);
    }
    SDD_CK(cudaEventRecord(p->ev[2 * slot], p->stream));
    SDD_TRY(launch_mc_round(p, false, nullptr, nullptr, nullptr, 0, 0));
    SDD_CK(cudaEventRecord(p->ev[2 * slot + 1], p->stream));
    return SDD_OK;
}

// Interface Monte Carlo of the nodes [lo, hi) (hi < 0: all M); the other nodes take no paths and
// their outputs are not meaningful.
sdd_status run_mc(sdd_problem* p, int lo = 0, int hi = -1)
{
    const TraceRange trace("sdd: interface Monte Carlo");
    const int M = p->M;
    p->stats.mc_rounds = 0;
    p->stats.mc_kernel_ms = 0.0;
    p->stats.mc_kernel_launches = 0;
    p->stats.path_steps = 0;
    p->stats.paths = 0;
    p->stats.nodes_not_reached = 0;
    p->stats.max_se = 0.0;
    if (M == 0) {
        SDD_CK(cudaMemcpyAsync(p->h_n_active + 1, p->bad, 4, cudaMemcpyDeviceToHost, p->stream));
        SDD_CK(cudaStreamSynchronize(p->stream));
        if (p->h_n_active[1]) return fail(SDD_ERR_INVALID_ARG, "monitor must be finite and > 0, mesh finite");
        p->have_est = true;
        return SDD_OK;
    }
    const bool adaptive = p->prm.se_target > 0;
    const int64_t n0 = p->prm.paths_per_node;
    const int64_t maxp = adaptive ? p->prm.max_paths_per_node : n0;
    if (hi < 0) hi = M;
    SDD_CK(launch_mc_init(M, n0, maxp, p->acc, p->n_done, p->steps, p->paths_run, p->next_total, p->stream,
                          p->n_interp > 0 ? p->iface_role : nullptr, lo, hi));
    p->launches += 1;
    int n_timed = 0;
    PlanParams PP{};
    PP.M = M; PP.n_done = p->n_done; PP.next_total = p->next_total; PP.node_of = p->node_of;
    PP.p_begin = p->p_begin; PP.p_count = p->p_count; PP.task_off = p->task_off;
    PP.n_active = p->n_active; PP.task_counter = p->task_counter;
    PP.task_paths = p->task_paths;
    ReduceParams RP{};
    RP.node_of = p->node_of; RP.p_count = p->p_count; RP.task_off = p->task_off;
    RP.n_active = p->n_active; RP.slots = p->slots; RP.shift = p->shift; RP.acc = p->acc;
    RP.n_done = p->n_done; RP.steps = p->steps; RP.paths_run = p->paths_run;
    RP.next_total = p->next_total; RP.se_target = adaptive ? p->prm.se_target : 0.0;
    RP.max_paths = maxp;
    if (!adaptive) {
        // fixed N: the number of launches is known, no host round trip
        const int64_t chunk = (int64_t)kTasksPerRound * p->task_paths;
        const int64_t rounds = (n0 + chunk - 1) / chunk;
        for (int64_t r = 0; r < rounds; ++r) {
            SDD_CK(launch_plan(PP, p->stream));
            SDD_TRY(timed_mc_round(p, n_timed++));
            SDD_CK(launch_reduce(RP, M, p->stream));
            p->launches += 3;
        }
        p->stats.mc_rounds = (int32_t)rounds;
    } else {
        // Rounds run kRoundsAhead ahead of the host's decision: rounds r+1 .. r+kRoundsAhead are
        // queued before the host reads round r's count of active nodes, so the GPU does not wait
        // on the host's round trip even when the host thread is slow to wake.  A round queued
        // after the last one with work finds no pending node; its plan, path kernel and
        // reduction change nothing.
        int queued = 0;
        for (int r = 0; r < kMaxAdaptiveRounds; ++r) {
            for (; queued < kMaxAdaptiveRounds && queued <= r + kRoundsAhead; ++queued) {
                const int slot = queued % (kRoundsAhead + 1);
                SDD_CK(launch_plan(PP, p->stream));
                SDD_CK(cudaMemcpyAsync(p->h_n_active + 2 + slot, p->n_active, sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, p->stream));
                SDD_CK(cudaEventRecord(p->count_ev[slot], p->stream));
                SDD_TRY(timed_mc_round(p, n_timed++));
                SDD_CK(launch_reduce(RP, M, p->stream));
                p->launches += 3;
            }
            const int slot = r % (kRoundsAhead + 1);
            SDD_CK(cudaEventSynchronize(p->count_ev[slot]));
            if (p->h_n_active[2 + slot] == 0) break;
            p->stats.mc_rounds = r + 1;
        }
    }
    SDD_CK(launch_output(M, p->acc, p->n_done, p->shift, p->est, p->se, p->stream));
    p->launches += 1;
    if (p->n_interp > 0) {
        SDD_CK(launch_interp(p->interp, p->n_interp, p->est, p->se, p->stream));
        p->launches += 1;
    }
    // counters (small copies)
    std::vector<int64_t> st(M), np(M);
    std::vector<double> se((size_t)2 * M);
    SDD_CK(cudaMemcpyAsync(st.data(), p->steps, 8 * (size_t)M, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(np.data(), p->paths_run, 8 * (size_t)M, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(se.data(), p->se, 16 * (size_t)M, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(p->h_n_active + 1, p->bad, 4, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaStreamSynchronize(p->stream));
    if (p->h_n_active[1]) return fail(SDD_ERR_INVALID_ARG, "monitor must be finite and > 0, mesh finite");
    p->stats.mc_kernel_ms = 0.0;
    p->stats.mc_kernel_launches = n_timed;
    for (int k = 0; k < n_timed; ++k) {
        float ms = 0.f;
        SDD_CK(cudaEventElapsedTime(&ms, p->ev[2 * k], p->ev[2 * k + 1]));
        p->stats.mc_kernel_ms += ms;
    }
    for (int m = lo; m < hi; ++m) {
        p->stats.path_steps += st[m];
        p->stats.paths += np[m];
        const double s = se[2 * m] > se[2 * m + 1] ? se[2 * m] : se[2 * m + 1];
        if (s > p->stats.max_se) p->stats.max_se = s;
        if (adaptive && s > p->prm.se_target) p->stats.nodes_not_reached += 1;
    }
    p->have_est = true;
    return p->stats.nodes_not_reached ? fail(SDD_ERR_SE_NOT_REACHED, "max_paths_per_node reached before se_target")
                                      : SDD_OK;
}

sdd_status run_solve(sdd_problem* p)
{
    const TraceRange trace("sdd: subdomain solves");
    SDD_CK(launch_scatter(p->prm.nx, p->prm.ny, p->prm.periodic, p->prm.Lx, p->prm.Ly, p->nodes, p->M,
                          p->est, p->xn, p->yn, p->stream, p->prm.moving_boundary ? p->bnd64 : nullptr));
    p->launches += (p->prm.periodic ? 0 : 1) + (p->M > 0 ? 1 : 0);
    SolveParams S{};
    S.nx = p->prm.nx; S.ny = p->prm.ny; S.px = p->prm.px; S.py = p->prm.py; S.form = p->prm.form;
    S.r = p->prm.dt / p->prm.tau; S.rtol = p->prm.solve_rtol; S.max_iter = p->prm.solve_max_iter;
    S.scheme = p->prm.subdomain_scheme;
    S.fe_max_substeps = p->prm.fe_max_substeps > 0 ? p->prm.fe_max_substeps : (1 << 16);
    S.om64 = p->om64; S.xcur = p->x; S.ycur = p->y; S.xnew = p->xn; S.ynew = p->yn;
    S.ce64 = p->ce64; S.cn64 = p->cn64; S.ce = p->ce; S.cn = p->cn; S.vec = p->vec;
    S.mg = p->mg; S.mg_stride = p->mg_stride;
    S.stat_iters = p->st_iters; S.stat_outer = p->st_outer; S.stat_ok = p->st_ok; S.stat_res = p->st_res;
    // device time of the solve launches
    if (!p->solve_ev[0]) SDD_CK(cudaEventCreate(&p->solve_ev[0]));
    if (!p->solve_ev[1]) SDD_CK(cudaEventCreate(&p->solve_ev[1]));
    SDD_CK(cudaEventRecord(p->solve_ev[0], p->stream));
    if (!p->h_items.empty())
        SDD_CK(launch_solve_items(S, p->solve_items, (int)p->h_items.size(), p->fp64, p->stream));
    else
        SDD_CK(launch_solve(S, p->fp64, p->stream));
    SDD_CK(cudaEventRecord(p->solve_ev[1], p->stream));
    p->launches += 2;
    const int ns = p->prm.px * p->prm.py;
    std::vector<int32_t> it(ns), ou(ns), ok(ns);
    std::vector<double> rs(ns);
    SDD_CK(cudaMemcpyAsync(it.data(), p->st_iters, 4 * (size_t)ns, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(ou.data(), p->st_outer, 4 * (size_t)ns, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(ok.data(), p->st_ok, 4 * (size_t)ns, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(rs.data(), p->st_res, 8 * (size_t)ns, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaStreamSynchronize(p->stream));
    p->stats.solve_iters_max = 0;
    p->stats.solve_outer_max = 0;
    p->stats.solve_rel_residual = 0.0;
    {
        float ms = 0.f;
        SDD_CK(cudaEventElapsedTime(&ms, p->solve_ev[0], p->solve_ev[1]));
        p->stats.solve_kernel_ms = ms;
    }
    int bad = 0;
    for (int s = 0; s < ns; ++s) {
        if (it[s] > p->stats.solve_iters_max) p->stats.solve_iters_max = it[s];
        if (ou[s] > p->stats.solve_outer_max) p->stats.solve_outer_max = ou[s];
        if (rs[s] > p->stats.solve_rel_residual) p->stats.solve_rel_residual = rs[s];
        bad += ok[s] ? 0 : 1;
    }
    return bad ? fail(SDD_ERR_NOT_CONVERGED, "a subdomain solve reached solve_max_iter") : SDD_OK;
}

// The new mesh becomes the current one; time and the step index advance.
sdd_status advance(sdd_problem* p, double* x_out, double* y_out)
{
    double* t;
    t = p->x; p->x = p->xn; p->xn = t;
    t = p->y; p->y = p->yn; p->yn = t;
    p->step += 1;
    p->have_est = false;
    p->stats.step_index = (int32_t)p->step;
    p->stats.t = p->prm.t0 + (double)p->step * p->prm.dt;
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_out(p, x_out, p->x, N * 8));
    SDD_TRY(copy_out(p, y_out, p->y, N * 8));
    return SDD_OK;
}
}  // namespace

// ---- Problem allocation (shared with the batch and server translation units) -------------

namespace {

// Every device array of a problem in allocation order; with_mc adds the problem's own interface
// Monte Carlo state (node sums, round plan, task slots, estimates).  p->prm, p->M and
// p->slot_cap must be set.
template <typename F>
void problem_arrays(sdd_problem* p, bool with_mc, F&& f)
{
    const sdd_params& q = p->prm;
    const size_t N = (size_t)q.nx * q.ny;
    const size_t M = (size_t)p->M;
    const size_t rs = q.precision == SDD_FP64 ? 8 : 4;
    const int ns = q.px * q.py;
    f((void**)&p->x, N * 8); f((void**)&p->y, N * 8); f((void**)&p->xn, N * 8); f((void**)&p->yn, N * 8);
    f((void**)&p->om64, N * 8); f((void**)&p->wxi64, N * 8); f((void**)&p->weta64, N * 8);
    f((void**)&p->omega_nodal, N * 8);
    f((void**)&p->mon, mon_bytes(q.nx, q.ny, q.precision == SDD_FP64)); f((void**)&p->disp, N * 2 * rs);
    f((void**)&p->nodes, (M + 1) * sizeof(int2));
    f((void**)&p->iface_role, (M + 1) * 4);
    f((void**)&p->interp, (size_t)(p->n_interp > 0 ? p->n_interp : 1) * sizeof(InterpRule));
    if (with_mc) {
        f((void**)&p->shift, (M + 1) * 16);
        f((void**)&p->acc, (M + 1) * 32); f((void**)&p->n_done, (M + 1) * 8); f((void**)&p->steps, (M + 1) * 8);
        f((void**)&p->paths_run, (M + 1) * 8); f((void**)&p->next_total, (M + 1) * 8);
        f((void**)&p->node_of, (M + 1) * 4); f((void**)&p->p_begin, (M + 1) * 8); f((void**)&p->p_count, (M + 1) * 8);
        f((void**)&p->task_off, (M + 2) * 8); f((void**)&p->n_active, 16); f((void**)&p->task_counter, 16);
        f((void**)&p->slots, (size_t)p->slot_cap * sizeof(TaskSlot));
        f((void**)&p->est, (M + 1) * 16); f((void**)&p->se, (M + 1) * 16);
    }
    f((void**)&p->ce64, N * 8); f((void**)&p->cn64, N * 8); f((void**)&p->ce, N * rs); f((void**)&p->cn, N * rs);
    f((void**)&p->vec, N * 4 * 2 * rs);
    f((void**)&p->st_iters, (size_t)ns * 4); f((void**)&p->st_outer, (size_t)ns * 4);
    f((void**)&p->st_ok, (size_t)ns * 4); f((void**)&p->st_res, (size_t)ns * 8);
    f((void**)&p->quality, (N + 2) * 8);
    f((void**)&p->mg, p->mg_stride * ns);
    f((void**)&p->bad, 16);
    f((void**)&p->solve_items, (p->h_items.size() + 1) * sizeof(SolveItem));
    const size_t nb = 2 * (size_t)q.nx + 2 * (size_t)q.ny;
    f((void**)&p->bnd64, nb * 8);
    f((void**)&p->bnd, nb * rs);
    f((void**)&p->bnd_scratch, 2 * nb * 8);
}

// Problem shell: parameters, interface layout, sizes; no device memory yet.
sdd_problem* problem_shell(const sdd_params& prm, cudaStream_t stream)
{
    sdd_problem* p = new sdd_problem();
    p->prm = prm;
    p->stream = stream;
    p->fp64 = prm.precision == SDD_FP64;
    p->acc_mode = prm.precision == SDD_FP32_KAHAN ? kAccKahan32 : kAcc64;
    layout(prm.nx, prm.ny, prm.px, prm.py, prm.periodic, p->ij);
    p->M = (int)(p->ij.size() / 2);
    sampling_table(prm, p->ij, p->h_role, p->h_interp);
    p->n_interp = (int)p->h_interp.size();
    p->slot_cap = (int64_t)(p->M > 0 ? p->M : 1) * kSlotsPerNode;
    const size_t rs = p->fp64 ? 8 : 4;
    // workspace slot per subdomain: the largest hierarchy over the subdomain widths, which are
    // floor((n-1)/P) or that plus one in each direction
    size_t mg = 0;
    const int wx = (prm.nx - 1) / prm.px, wy = (prm.ny - 1) / prm.py;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const size_t m = mg_bytes(wx + a - 1, wy + b - 1, rs);
            if (m > mg) mg = m;
        }
    p->mg_stride = mg;
    // subdomains by interior size, largest first; large ones are solved by a cluster of CTAs
    std::vector<std::pair<int64_t, int2>> subs;
    for (int k = 0; k < prm.px * prm.py; ++k) {
        const int I = k % prm.px, J = k / prm.px;
        const int64_t wi = split_line(I + 1, prm.nx, prm.px) - split_line(I, prm.nx, prm.px) - 1;
        const int64_t wj = split_line(J + 1, prm.ny, prm.py) - split_line(J, prm.ny, prm.py) - 1;
        subs.push_back({wi * wj, make_int2(0, k)});
    }
    std::stable_sort(subs.begin(), subs.end(), [](const std::pair<int64_t, int2>& a,
                                                  const std::pair<int64_t, int2>& c) { return a.first > c.first; });
    if (prm.subdomain_scheme == 0) p->h_items = solve_items(subs);
    p->stats.M = p->M;
    p->stats.t = prm.t0;
    return p;
}

size_t alloc_rounded(size_t bytes) { return ((bytes < 16 ? 16 : bytes) + 511) / 512 * 512; }

}  // namespace

sdd_status sdd_validate_params(const sdd_params* P) { return validate(P); }

void sdd_layout(int nx, int ny, int px, int py, int periodic, std::vector<int32_t>& ij)
{
    layout(nx, ny, px, py, periodic, ij);
}

size_t sdd_problem_device_bytes(const sdd_params& prm, bool with_mc)
{
    sdd_problem* p = problem_shell(prm, nullptr);
    size_t total = 0;
    problem_arrays(p, with_mc, [&](void**, size_t b) { total += alloc_rounded(b); });
    delete p;
    return total;
}

sdd_status sdd_alloc_problem(const sdd_params& prm, cudaStream_t stream, bool with_mc, sdd_problem** out)
{
    *out = nullptr;
    sdd_problem* p = problem_shell(prm, stream);
    cudaError_t e = cudaSuccess;
    problem_arrays(p, with_mc, [&](void** ptr, size_t b) {
        if (e == cudaSuccess) e = p->dalloc(ptr, b);
        if (e == cudaSuccess) p->dev_bytes += alloc_rounded(b);
    });
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&p->h_n_active, 32, cudaHostAllocDefault);
    for (int k = 0; k <= kRoundsAhead && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&p->count_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const std::string msg = std::string("allocation failed: ") + cudaGetErrorString(e);
        delete p;
        return fail(e == cudaErrorMemoryAllocation ? SDD_ERR_OOM : SDD_ERR_CUDA, msg);
    }
    const size_t N = (size_t)prm.nx * prm.ny;
    const size_t rs = p->fp64 ? 8 : 4;
    e = cudaMemsetAsync(p->vec, 0, N * 4 * 2 * rs, p->stream);
    if (e == cudaSuccess && p->M > 0)
        e = cudaMemcpyAsync(p->nodes, p->ij.data(), (size_t)p->M * sizeof(int2), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess && p->M > 0)
        e = cudaMemcpyAsync(p->iface_role, p->h_role.data(), (size_t)p->M * 4, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess && p->n_interp > 0)
        e = cudaMemcpyAsync(p->interp, p->h_interp.data(), (size_t)p->n_interp * sizeof(InterpRule),
                            cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess && !p->h_items.empty())
        e = cudaMemcpyAsync(p->solve_items, p->h_items.data(), p->h_items.size() * sizeof(SolveItem),
                            cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);  // p->ij is pageable host memory
    if (e != cudaSuccess) {
        cudaGetLastError();
        const std::string msg = std::string("problem setup: ") + cudaGetErrorString(e);
        delete p;
        return fail(SDD_ERR_CUDA, msg);
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = p->fp64 ? mc_max_blocks_per_sm<double>(p->acc_mode, false, false)
                               : mc_max_blocks_per_sm<float>(p->acc_mode, false, false);
    p->nsm = nsm;
    p->mc_max_blocks_per_sm = per_sm;
    p->mc_blocks_per_sm = per_sm;
    p->mc_grid = nsm * per_sm;
    *out = p;
    return SDD_OK;
}

bool sdd_boundary_ok(const sdd_params& prm, const double* hx, const double* hy)
{
    if (prm.periodic) return true;
    const int nx = prm.nx, ny = prm.ny;
    const double tol = 1e-12 * (prm.Lx + prm.Ly);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (i != 0 && j != 0 && i != nx - 1 && j != ny - 1) continue;
            const double bx = prm.Lx * ((double)i / (double)(nx - 1));
            const double by = prm.Ly * ((double)j / (double)(ny - 1));
            const size_t id = (size_t)j * nx + i;
            if (prm.moving_boundary) {  // only the normal components are fixed
                if ((i == 0 || i == nx - 1) && !(fabs(hx[id] - bx) <= tol)) return false;
                if ((j == 0 || j == ny - 1) && !(fabs(hy[id] - by) <= tol)) return false;
                continue;
            }
            if (!(fabs(hx[id] - bx) <= tol) || !(fabs(hy[id] - by) <= tol)) return false;
        }
    return true;
}

extern "C" {

const char* sdd_status_string(sdd_status s)
{
    switch (s) {
    case SDD_OK: return "ok";
    case SDD_ERR_INVALID_ARG: return "invalid argument";
    case SDD_ERR_OOM: return "out of memory";
    case SDD_ERR_CUDA: return "CUDA error";
    case SDD_ERR_NOT_CONVERGED: return "subdomain solve not converged";
    case SDD_ERR_SE_NOT_REACHED: return "standard-error target not reached";
    case SDD_ERR_NO_DEVICE: return "no CUDA device";
    case SDD_ERR_CANCELLED: return "request cancelled";
    }
    return "unknown status";
}

const char* sdd_last_error(void) { return g_err.c_str(); }

sdd_status sdd_interface_layout(int32_t nx, int32_t ny, int32_t px, int32_t py, int32_t periodic,
                                int32_t* ij, int32_t* M)
{
    if (!M) return fail(SDD_ERR_INVALID_ARG, "M is NULL");
    if (nx < 3 || ny < 3 || px < 1 || py < 1 || px > nx - 1 || py > ny - 1 || (periodic != 0 && periodic != 1))
        return fail(SDD_ERR_INVALID_ARG, "bad grid or split");
    std::vector<int32_t> v;
    layout(nx, ny, px, py, periodic, v);
    *M = (int32_t)(v.size() / 2);
    if (ij && !v.empty()) memcpy(ij, v.data(), v.size() * sizeof(int32_t));
    return SDD_OK;
}

sdd_status sdd_interface_sampling(const sdd_params* params, int32_t* sampled, int32_t* M)
{
    if (!M) return fail(SDD_ERR_INVALID_ARG, "M is NULL");
    SDD_TRY(validate(params));
    std::vector<int32_t> ij, role;
    std::vector<InterpRule> rules;
    layout(params->nx, params->ny, params->px, params->py, params->periodic, ij);
    sampling_table(*params, ij, role, rules);
    *M = (int32_t)role.size();
    if (sampled)
        for (size_t m = 0; m < role.size(); ++m) sampled[m] = role[m] < 0 ? 1 : 0;
    return SDD_OK;
}

int64_t sdd_adaptive_next_total(int64_t n_done, double se, double target, int64_t max_paths)
{
    return adaptive_next_total(n_done, se, target, max_paths);
}

sdd_status sdd_create_problem(const sdd_params* params, const double* x0, const double* y0, void* stream,
                              sdd_problem** out)
{
    if (!out) return fail(SDD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    SDD_TRY(validate(params));
    if (!x0 || !y0) return fail(SDD_ERR_INVALID_ARG, "x0, y0 must not be NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SDD_ERR_NO_DEVICE, "no CUDA device visible");
    }
    sdd_problem* p = nullptr;
    SDD_TRY(sdd_alloc_problem(*params, static_cast<cudaStream_t>(stream), true, &p));
    auto bail = [&](sdd_status s) { delete p; return s; };
    {
        sdd_status s = check_boundary(p, x0, y0);
        if (s != SDD_OK) return bail(s);
    }
    const size_t N = (size_t)params->nx * params->ny;
    auto ck = [&](cudaError_t c, const char* what) -> sdd_status {
        if (c == cudaSuccess) return SDD_OK;
        return fail(SDD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(c));
    };
    sdd_status s = SDD_OK;
    if (s == SDD_OK) s = ck(cudaMemcpyAsync(p->x, x0, N * 8, cudaMemcpyDefault, p->stream), "copy x0");
    if (s == SDD_OK) s = ck(cudaMemcpyAsync(p->y, y0, N * 8, cudaMemcpyDefault, p->stream), "copy y0");
    // default monitor: omega = 1 everywhere
    if (s == SDD_OK) {
        std::vector<double> ones(N, 1.0);
        s = ck(cudaMemcpyAsync(p->omega_nodal, ones.data(), N * 8, cudaMemcpyHostToDevice, p->stream), "copy omega");
        if (s == SDD_OK) s = ck(cudaStreamSynchronize(p->stream), "sync");
    }
    if (s != SDD_OK) return bail(s);
    *out = p;
    return SDD_OK;
}

void sdd_destroy_problem(sdd_problem* p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    delete p;
}

sdd_status sdd_set_stream(sdd_problem* p, void* stream)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    SDD_CK(cudaStreamSynchronize(p->stream));
    p->stream = static_cast<cudaStream_t>(stream);
    return SDD_OK;
}

sdd_status sdd_set_mesh(sdd_problem* p, const double* x, const double* y)
{
    if (!p || !x || !y) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    SDD_TRY(check_boundary(p, x, y));
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_in(p, p->x, x, N * 8));
    SDD_TRY(copy_in(p, p->y, y, N * 8));
    p->have_est = false;
    return SDD_OK;
}

sdd_status sdd_get_mesh(sdd_problem* p, double* x, double* y)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_out(p, x, p->x, N * 8));
    SDD_TRY(copy_out(p, y, p->y, N * 8));
    return SDD_OK;
}

sdd_status sdd_set_monitor(sdd_problem* p, const double* omega)
{
    if (!p || !omega) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_in(p, p->omega_nodal, omega, N * 8));
    p->mon_kind = SDD_MONITOR_NODAL;
    p->n_params = 0;
    return SDD_OK;
}

sdd_status sdd_set_monitor_analytic(sdd_problem* p, int32_t kind, const double* params, int32_t n_params)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    if (kind == SDD_MONITOR_GAUSS && n_params != 4) return fail(SDD_ERR_INVALID_ARG, "GAUSS needs 4 params");
    if (kind == SDD_MONITOR_FRONT && n_params != 6) return fail(SDD_ERR_INVALID_ARG, "FRONT needs 6 params");
    if (kind == SDD_MONITOR_BUMPS && (n_params % 4 || n_params < 0 || n_params > 64))
        return fail(SDD_ERR_INVALID_ARG, "BUMPS needs 4k params, k <= 16");
    if (kind == SDD_MONITOR_RINGS && (n_params < 5 || (n_params - 3) % 2 || n_params > 63))
        return fail(SDD_ERR_INVALID_ARG, "RINGS needs 3 + 2k params, 1 <= k <= 30");
    if (kind < SDD_MONITOR_GAUSS || kind > SDD_MONITOR_RINGS) return fail(SDD_ERR_INVALID_ARG, "bad monitor kind");
    if (n_params > 0 && !params) return fail(SDD_ERR_INVALID_ARG, "params is NULL");
    p->mon_kind = kind;
    p->n_params = n_params;
    memset(p->mon_params, 0, sizeof(p->mon_params));
    for (int k = 0; k < n_params; ++k) p->mon_params[k] = params[k];
    return SDD_OK;
}

sdd_status sdd_interface_mc(sdd_problem* p, double* est_xy, double* se_xy, int64_t* paths_used)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    SDD_TRY(run_prep(p));
    const sdd_status s = run_mc(p);
    if (s != SDD_OK && s != SDD_ERR_SE_NOT_REACHED) return s;
    const size_t M = (size_t)p->M;
    SDD_TRY(copy_out(p, est_xy, p->est, M * 16));
    SDD_TRY(copy_out(p, se_xy, p->se, M * 16));
    SDD_TRY(copy_out(p, paths_used, p->n_done, M * 8));
    return s;
}

sdd_status sdd_subdomain_solve(sdd_problem* p, const double* iface_xy, double* x_out, double* y_out)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    SDD_TRY(run_prep(p));
    if (iface_xy) {
        SDD_TRY(copy_in(p, p->est, iface_xy, (size_t)p->M * 16));
        p->have_est = true;
    }
    if (!p->have_est) return fail(SDD_ERR_INVALID_ARG, "no interface data: pass iface_xy or call sdd_interface_mc");
    const sdd_status s = run_solve(p);
    if (s != SDD_OK && s != SDD_ERR_NOT_CONVERGED) return s;
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_out(p, x_out, p->xn, N * 8));
    SDD_TRY(copy_out(p, y_out, p->yn, N * 8));
    return s;
}

sdd_status sdd_step(sdd_problem* p, double* x_out, double* y_out)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    const TraceRange trace("sdd_step");
    SDD_TRY(run_prep(p));
    const sdd_status s_mc = run_mc(p);
    if (s_mc != SDD_OK && s_mc != SDD_ERR_SE_NOT_REACHED) return s_mc;
    const sdd_status s_sv = run_solve(p);
    if (s_sv != SDD_OK && s_sv != SDD_ERR_NOT_CONVERGED) return s_sv;
    SDD_TRY(advance(p, x_out, y_out));
    if (s_mc != SDD_OK) return fail(s_mc, "max_paths_per_node reached before se_target");
    return s_sv;
}

sdd_status sdd_interface_mc_range(sdd_problem* p, int32_t node_begin, int32_t node_end, double* est_xy,
                                  double* se_xy, int64_t* paths_used)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    if (node_begin < 0 || node_end < node_begin || node_end > p->M)
        return fail(SDD_ERR_INVALID_ARG, "node range outside [0, M]");
    if (p->n_interp > 0)
        return fail(SDD_ERR_INVALID_ARG, "interface sampling: interpolated nodes need the estimates of every range");
    SDD_TRY(run_prep(p));
    if (node_end == node_begin) return SDD_OK;
    const sdd_status s = run_mc(p, node_begin, node_end);
    if (s != SDD_OK && s != SDD_ERR_SE_NOT_REACHED) return s;
    const size_t b = (size_t)node_begin, n = (size_t)(node_end - node_begin);
    SDD_TRY(copy_out(p, est_xy ? est_xy + 2 * b : nullptr, p->est + 2 * b, n * 16));
    SDD_TRY(copy_out(p, se_xy ? se_xy + 2 * b : nullptr, p->se + 2 * b, n * 16));
    SDD_TRY(copy_out(p, paths_used ? paths_used + b : nullptr, p->n_done + b, n * 8));
    p->have_est = false;  // the problem's own estimates cover this range only
    return s;
}

sdd_status sdd_step_from_interface(sdd_problem* p, const double* iface_xy, double* x_out, double* y_out)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    if (!iface_xy && p->M > 0) return fail(SDD_ERR_INVALID_ARG, "iface_xy is NULL");
    SDD_TRY(run_prep(p));
    if (p->M > 0) SDD_TRY(copy_in(p, p->est, iface_xy, (size_t)p->M * 16));
    const sdd_status s_sv = run_solve(p);
    if (s_sv != SDD_OK && s_sv != SDD_ERR_NOT_CONVERGED) return s_sv;
    SDD_TRY(advance(p, x_out, y_out));
    return s_sv;
}

sdd_status sdd_step_mkp(sdd_problem* p, int32_t K, double* x_out, double* y_out)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    if (K < 1 || K > (1 << 16)) return fail(SDD_ERR_INVALID_ARG, "K must be in [1, 2^16]");
    const int64_t n = p->step;
    if ((n + 1) * (int64_t)K > ((int64_t)1 << 32))
        return fail(SDD_ERR_INVALID_ARG, "time-step word n K + k exceeds 32 bits");
    const sdd_params saved = p->prm;
    p->prm.dt = saved.dt / (double)K;
    p->t_monitor = saved.t0 + (double)n * saved.dt;
    p->monitor_time_fixed = true;
    sdd_status hard = SDD_OK, soft = SDD_OK;
    sdd_stats acc{};
    int k = 0;
    for (; k < K; ++k) {
        p->step = n * K + k;
        hard = run_prep(p);
        if (hard != SDD_OK) break;
        const sdd_status s_mc = run_mc(p);
        if (s_mc != SDD_OK && s_mc != SDD_ERR_SE_NOT_REACHED) { hard = s_mc; break; }
        const sdd_status s_sv = run_solve(p);
        if (s_sv != SDD_OK && s_sv != SDD_ERR_NOT_CONVERGED) { hard = s_sv; break; }
        if (soft == SDD_OK) soft = s_mc != SDD_OK ? s_mc : s_sv;
        double* t;
        t = p->x; p->x = p->xn; p->xn = t;
        t = p->y; p->y = p->yn; p->yn = t;
        acc.path_steps += p->stats.path_steps;
        acc.paths += p->stats.paths;
        acc.mc_rounds += p->stats.mc_rounds;
        acc.mc_kernel_ms += p->stats.mc_kernel_ms;
        acc.mc_kernel_launches += p->stats.mc_kernel_launches;
        acc.nodes_not_reached += p->stats.nodes_not_reached;
        if (p->stats.max_se > acc.max_se) acc.max_se = p->stats.max_se;
        if (p->stats.solve_iters_max > acc.solve_iters_max) acc.solve_iters_max = p->stats.solve_iters_max;
        if (p->stats.solve_outer_max > acc.solve_outer_max) acc.solve_outer_max = p->stats.solve_outer_max;
        if (p->stats.solve_rel_residual > acc.solve_rel_residual) acc.solve_rel_residual = p->stats.solve_rel_residual;
    }
    p->prm = saved;
    p->monitor_time_fixed = false;
    p->have_est = false;
    if (hard != SDD_OK) {
        // the mesh is the last completed sub-mesh; the step index stays n
        p->step = n;
        p->stats.step_index = (int32_t)n;
        return hard;
    }
    p->step = n + 1;
    p->stats.path_steps = acc.path_steps;
    p->stats.paths = acc.paths;
    p->stats.mc_rounds = acc.mc_rounds;
    p->stats.mc_kernel_ms = acc.mc_kernel_ms;
    p->stats.mc_kernel_launches = acc.mc_kernel_launches;
    p->stats.nodes_not_reached = acc.nodes_not_reached;
    p->stats.max_se = acc.max_se;
    p->stats.solve_iters_max = acc.solve_iters_max;
    p->stats.solve_outer_max = acc.solve_outer_max;
    p->stats.solve_rel_residual = acc.solve_rel_residual;
    p->stats.step_index = (int32_t)p->step;
    p->stats.t = p->prm.t0 + (double)p->step * p->prm.dt;
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_out(p, x_out, p->x, N * 8));
    SDD_TRY(copy_out(p, y_out, p->y, N * 8));
    if (soft == SDD_ERR_SE_NOT_REACHED) return fail(soft, "max_paths_per_node reached before se_target");
    if (soft == SDD_ERR_NOT_CONVERGED) return fail(soft, "a subdomain solve reached solve_max_iter");
    return SDD_OK;
}

sdd_status sdd_get_stats(const sdd_problem* p, sdd_stats* out)
{
    if (!p || !out) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    *out = p->stats;
    out->kernel_launches = p->launches;
    out->M = p->M;
    out->step_index = (int32_t)p->step;
    out->t = p->prm.t0 + (double)p->step * p->prm.dt;
    return SDD_OK;
}

sdd_status sdd_get_mc_config(const sdd_problem* p, sdd_mc_config* out)
{
    if (!p || !out) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    out->threads_per_block = 256;
    out->blocks_per_sm = p->mc_blocks_per_sm;
    out->paths_per_task = p->task_paths;
    out->max_blocks_per_sm = p->mc_max_blocks_per_sm;
    return SDD_OK;
}

sdd_status sdd_set_mc_config(sdd_problem* p, const sdd_mc_config* c)
{
    if (!p || !c) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (c->threads_per_block != 0 && c->threads_per_block != 256)
        return fail(SDD_ERR_INVALID_ARG, "a single problem's path kernel runs 256 threads per block");
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > p->mc_max_blocks_per_sm)
        return fail(SDD_ERR_INVALID_ARG, "blocks_per_sm must be in [0, max_blocks_per_sm]");
    if (c->paths_per_task != 0 && !sdd_valid_task_paths(c->paths_per_task))
        return fail(SDD_ERR_INVALID_ARG, "paths_per_task must be 1024, 2048 or 4096");
    if (c->paths_per_task) p->task_paths = c->paths_per_task;
    p->mc_blocks_per_sm = c->blocks_per_sm ? c->blocks_per_sm : p->mc_max_blocks_per_sm;
    p->mc_grid = p->nsm * p->mc_blocks_per_sm;
    return SDD_OK;
}

sdd_status sdd_tune(sdd_problem* p, int32_t tune_paths_per_task, sdd_mc_config* chosen)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    if (tune_paths_per_task != 0 && tune_paths_per_task != 1)
        return fail(SDD_ERR_INVALID_ARG, "tune_paths_per_task must be 0 or 1");
    const TraceRange trace("sdd_tune");
    SDD_CK(cudaStreamSynchronize(p->stream));
    if (p->M > 0) {
        SDD_TRY(run_prep(p));
        const int64_t n0 = p->prm.paths_per_node;
        const int64_t maxp = p->prm.se_target > 0 ? p->prm.max_paths_per_node : n0;
        SDD_CK(launch_mc_init(p->M, n0, maxp, p->acc, p->n_done, p->steps, p->paths_run, p->next_total,
                              p->stream, p->n_interp > 0 ? p->iface_role : nullptr));
        p->launches += 1;
        PlanParams PP{};
        PP.M = p->M; PP.n_done = p->n_done; PP.next_total = p->next_total; PP.node_of = p->node_of;
        PP.p_begin = p->p_begin; PP.p_count = p->p_count; PP.task_off = p->task_off;
        PP.n_active = p->n_active; PP.task_counter = p->task_counter;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        SDD_CK(cudaEventCreate(&e0));
        cudaError_t ce = cudaEventCreate(&e1);
        const int tps[3] = {1024, 2048, 4096};
        const int nt = tune_paths_per_task ? 3 : 1;
        double best = -1.0;
        int best_t = p->task_paths, best_b = p->mc_blocks_per_sm;
        for (int a = 0; a < nt && ce == cudaSuccess; ++a) {
            const int T = tune_paths_per_task ? tps[a] : p->task_paths;
            // paths of the round at this task size (a round gives a node at most 256 tasks)
            const int64_t round = n0 < (int64_t)kTasksPerRound * T ? n0 : (int64_t)kTasksPerRound * T;
            PP.task_paths = T;
            for (int bps = 1; bps <= p->mc_max_blocks_per_sm && ce == cudaSuccess; ++bps) {
                float ms_min = 0.f;
                for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {
                    ce = launch_plan(PP, p->stream);
                    if (ce == cudaSuccess) ce = cudaEventRecord(e0, p->stream);
                    if (ce != cudaSuccess) break;
                    if (p->fp64) {
                        McParams<double> P = mc_params<double>(p);
                        P.task_paths = T;
                        ce = launch_mc<double>(P, p->acc_mode, false, false, p->nsm * bps, p->stream);
                    } else {
                        McParams<float> P = mc_params<float>(p);
                        P.task_paths = T;
                        ce = launch_mc<float>(P, p->acc_mode, false, false, p->nsm * bps, p->stream);
                    }
                    if (ce == cudaSuccess) ce = cudaEventRecord(e1, p->stream);
                    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                    if (ce == cudaSuccess && (rep == 0 || ms < ms_min)) ms_min = ms;
                    p->launches += 2;
                }
                const double per_path = (double)ms_min / (double)round;
                if (ce == cudaSuccess && (best < 0 || per_path < best)) {
                    best = per_path;
                    best_t = T;
                    best_b = bps;
                }
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(SDD_ERR_CUDA, cudaGetErrorString(ce));
        }
        p->task_paths = best_t;
        p->mc_blocks_per_sm = best_b;
        p->mc_grid = p->nsm * best_b;
    }
    return chosen ? sdd_get_mc_config(p, chosen) : SDD_OK;
}

sdd_status sdd_get_interface_nodes(const sdd_problem* p, int32_t* ij, int32_t* M)
{
    if (!p || !M) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    *M = p->M;
    if (ij && p->M > 0) memcpy(ij, p->ij.data(), p->ij.size() * sizeof(int32_t));
    return SDD_OK;
}

sdd_status sdd_save(sdd_problem* p, const char* path)
{
    if (!p || !path) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    std::vector<double> buf(3 * N);
    SDD_CK(cudaMemcpyAsync(buf.data(), p->x, N * 8, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(buf.data() + N, p->y, N * 8, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaMemcpyAsync(buf.data() + 2 * N, p->omega_nodal, N * 8, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaStreamSynchronize(p->stream));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(SDD_ERR_INVALID_ARG, std::string("cannot write ") + path);
    const int32_t rec = (int32_t)sizeof(sdd_params);
    const int64_t step = p->step;
    const int32_t kind = p->mon_kind, np = p->n_params;
    bool ok = fwrite(kCkptMagic, 1, 8, f) == 8 && fwrite(&rec, 4, 1, f) == 1 &&
              fwrite(&p->prm, sizeof(sdd_params), 1, f) == 1 && fwrite(&step, 8, 1, f) == 1 &&
              fwrite(&kind, 4, 1, f) == 1 && fwrite(&np, 4, 1, f) == 1 &&
              fwrite(p->mon_params, 8, 64, f) == 64 && fwrite(buf.data(), 8, 3 * N, f) == 3 * N;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(SDD_ERR_INVALID_ARG, std::string("short write to ") + path);
    return SDD_OK;
}

sdd_status sdd_load(const char* path, void* stream, sdd_problem** out)
{
    if (!path || !out) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(SDD_ERR_INVALID_ARG, std::string("cannot read ") + path);
    char magic[8];
    int32_t rec = 0, kind = 0, np = 0;
    int64_t step = 0;
    sdd_params prm{};
    double mp[64];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kCkptMagic, 8) == 0 && fread(&rec, 4, 1, f) == 1 &&
              rec == (int32_t)sizeof(sdd_params) && fread(&prm, sizeof(sdd_params), 1, f) == 1 &&
              fread(&step, 8, 1, f) == 1 && fread(&kind, 4, 1, f) == 1 && fread(&np, 4, 1, f) == 1 &&
              fread(mp, 8, 64, f) == 64;
    std::vector<double> buf;
    if (ok) ok = validate(&prm) == SDD_OK && step >= 0 && step < ((int64_t)1 << 32) && kind >= SDD_MONITOR_NODAL &&
                 kind <= SDD_MONITOR_RINGS && np >= 0 && np <= 64;
    if (ok) {
        const size_t N = (size_t)prm.nx * prm.ny;
        buf.resize(3 * N);
        ok = fread(buf.data(), 8, 3 * N, f) == 3 * N && fgetc(f) == EOF;
    }
    fclose(f);
    if (!ok) return fail(SDD_ERR_INVALID_ARG, std::string("not a valid checkpoint: ") + path);
    const size_t N = (size_t)prm.nx * prm.ny;
    sdd_problem* p = nullptr;
    SDD_TRY(sdd_create_problem(&prm, buf.data(), buf.data() + N, stream, &p));
    sdd_status s = SDD_OK;
    if (kind == SDD_MONITOR_NODAL) s = sdd_set_monitor(p, buf.data() + 2 * N);
    else s = sdd_set_monitor_analytic(p, kind, mp, np);
    if (s == SDD_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) s = fail(SDD_ERR_CUDA, "sync");
    if (s != SDD_OK) {
        delete p;
        return s;
    }
    p->step = step;
    p->stats.step_index = (int32_t)step;
    p->stats.t = prm.t0 + (double)step * prm.dt;
    *out = p;
    return SDD_OK;
}

sdd_status sdd_get_monitor(sdd_problem* p, double* omega, double* w_xi, double* w_eta)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    SDD_TRY(run_prep(p));
    const size_t N = (size_t)p->prm.nx * p->prm.ny;
    SDD_TRY(copy_out(p, omega, p->om64, N * 8));
    SDD_TRY(copy_out(p, w_xi, p->wxi64, N * 8));
    SDD_TRY(copy_out(p, w_eta, p->weta64, N * 8));
    SDD_CK(cudaStreamSynchronize(p->stream));
    return SDD_OK;
}

sdd_status sdd_mesh_quality(sdd_problem* p, double* q_cells, double* q_max, double* q_mean)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    const int nx = p->prm.nx, ny = p->prm.ny;
    const size_t nc = (size_t)(nx - 1) * (ny - 1);
    SDD_CK(launch_quality(nx, ny, p->x, p->y, p->quality, p->quality + nc, p->stream));
    p->launches += 2;
    double st[2] = {0.0, 0.0};
    SDD_TRY(copy_out(p, q_cells, p->quality, nc * 8));
    SDD_CK(cudaMemcpyAsync(st, p->quality + nc, 16, cudaMemcpyDeviceToHost, p->stream));
    SDD_CK(cudaStreamSynchronize(p->stream));
    if (q_max) *q_max = st[0];
    if (q_mean) *q_mean = st[1];
    return SDD_OK;
}

sdd_status sdd_debug_paths(sdd_problem* p, int32_t node, int64_t p_begin, int64_t n_paths, double* val_xy,
                           int32_t* exit_step, int8_t* exit_side)
{
    if (!p) return fail(SDD_ERR_INVALID_ARG, "problem is NULL");
    if (node < 0 || node >= p->M) return fail(SDD_ERR_INVALID_ARG, "node out of range");
    if (n_paths < 1 || p_begin < 0 || p_begin + n_paths > ((int64_t)1 << 32))
        return fail(SDD_ERR_INVALID_ARG, "path range out of [0, 2^32)");
    const int64_t tasks = (n_paths + p->task_paths - 1) / p->task_paths;
    if (tasks > p->slot_cap) return fail(SDD_ERR_INVALID_ARG, "too many paths for one debug call");
    SDD_TRY(run_prep(p));
    double* dval = nullptr;
    int32_t* dst = nullptr;
    int8_t* dsd = nullptr;
    SDD_CK(cudaMalloc(&dval, (size_t)n_paths * 16));
    cudaError_t e = cudaMalloc(&dst, (size_t)n_paths * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dsd, (size_t)n_paths);
    sdd_status s = SDD_OK;
    if (e != cudaSuccess) s = fail(SDD_ERR_OOM, "debug buffers");
    // one-node plan
    const int32_t h_node = node, h_act = 1, h_zero = 0;
    const int64_t h_off[2] = {0, tasks};
    auto ck = [&](cudaError_t c) {
        if (s == SDD_OK && c != cudaSuccess) s = fail(SDD_ERR_CUDA, cudaGetErrorString(c));
    };
    if (s == SDD_OK) {
        ck(cudaMemcpyAsync(p->node_of, &h_node, 4, cudaMemcpyHostToDevice, p->stream));
        ck(cudaMemcpyAsync(p->p_begin, &p_begin, 8, cudaMemcpyHostToDevice, p->stream));
        ck(cudaMemcpyAsync(p->p_count, &n_paths, 8, cudaMemcpyHostToDevice, p->stream));
        ck(cudaMemcpyAsync(p->task_off, h_off, 16, cudaMemcpyHostToDevice, p->stream));
        ck(cudaMemcpyAsync(p->n_active, &h_act, 4, cudaMemcpyHostToDevice, p->stream));
        ck(cudaMemcpyAsync(p->task_counter, &h_zero, 4, cudaMemcpyHostToDevice, p->stream));
    }
    if (s == SDD_OK) s = launch_mc_round(p, true, dval, dst, dsd, p_begin, n_paths);
    if (s == SDD_OK) s = copy_out(p, val_xy, dval, (size_t)n_paths * 16);
    if (s == SDD_OK) s = copy_out(p, exit_step, dst, (size_t)n_paths * 4);
    if (s == SDD_OK) s = copy_out(p, exit_side, dsd, (size_t)n_paths);
    if (s == SDD_OK) ck(cudaStreamSynchronize(p->stream));
    cudaFree(dval);
    if (dst) cudaFree(dst);
    if (dsd) cudaFree(dsd);
    return s;
}

sdd_status sdd_debug_unit_math(const uint32_t* w, int64_t n, float* out)
{
    if (n < 0 || (n > 0 && (!w || !out))) return fail(SDD_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return SDD_OK;
    uint32_t* dw = nullptr;
    float* dout = nullptr;
    SDD_CK(cudaMalloc(&dw, (size_t)n * 4));
    cudaError_t e = cudaMalloc(&dout, (size_t)n * 20);
    if (e == cudaSuccess) e = cudaMemcpy(dw, w, (size_t)n * 4, cudaMemcpyDefault);
    if (e == cudaSuccess) e = launch_unit_math(dw, n, dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)n * 20, cudaMemcpyDefault);
    cudaFree(dw);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(SDD_ERR_CUDA, cudaGetErrorString(e));
    return SDD_OK;
}

sdd_status sdd_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(SDD_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return SDD_OK;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    SDD_CK(cudaMalloc(&dc, (size_t)n * 16));
    cudaError_t e = cudaMalloc(&dk, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)n * 16);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, (size_t)n * 16, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, (size_t)n * 8, cudaMemcpyDefault);
    if (e == cudaSuccess) e = launch_philox(dc, dk, n, dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)n * 16, cudaMemcpyDefault);
    cudaFree(dc);
    if (dk) cudaFree(dk);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(SDD_ERR_CUDA, cudaGetErrorString(e));
    return SDD_OK;
}

}  // extern "C"
