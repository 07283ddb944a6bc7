// Allocation-free interface Monte Carlo: sdd_interface_mc_noalloc (declared in include/sdd.h).
//
// Some callers cannot call cudaMalloc: a host framework whose caching allocator owns the
// device memory budget and forbids allocations outside it, or a latency-critical loop that
// cannot afford a device allocation (and the synchronisation cudaMalloc/cudaFree may imply).
// This entry point runs the same kernels as sdd_interface_mc (fixed path count) without any
// allocation: the caller passes inputs and outputs in device memory, and every intermediate
// (monitor records, node list, node sums, round plan, task slots) lives in one file-scope
// device array of kScratchBytes.  Every GPU that loads the library holds that array until the
// process exits.  Calls share the array and it keeps the last call's contents: a call
// re-initialises everything it reads, and calls that overlap on the GPU race.
//
// The array's name in host code is a host-side stand-in, not a device address; its device
// address is resolved with cudaGetSymbolAddress on the first call made with a device current
// (make that first call before any stream capture), and again whenever that device's context
// has changed since (a cudaDeviceReset in between reloads the module at another address).
//
// Inputs are not checked on the device: omega must be finite and > 0, the mesh finite, and on
// Dirichlet grids the boundary the identity; otherwise the estimates are undefined.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sdd.h"
#include "sdd_internal.cuh"

namespace {

using namespace sdd;

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;
constexpr int64_t kMaxChunk = int64_t(1) << 19;     // paths per node per launch (plan kernel)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, with the unique id of the context it was
// resolved in (context ids are never reused within a process).
struct ScratchAddr {
    void* addr = nullptr;
    unsigned long long ctx_id = 0;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Unique id of the calling thread's current context (0 when there is none or the driver
// entry points are unavailable).  The driver functions are found through the runtime, so the
// library needs no link against the driver library.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

sdd_status scratch_for_current_device(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SDD_ERR_NO_DEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) return SDD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchAddr& c = g_scratch_addr[dev];
    const unsigned long long id = current_context_id();
    if (!c.addr || id == 0 || id != c.ctx_id) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // creates the context if needed
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            c = ScratchAddr{};
            return SDD_ERR_CUDA;
        }
        c.addr = p;
        c.ctx_id = current_context_id();
    }
    *out = c.addr;
    return SDD_OK;
}

// Bump allocator over the scratch array (base == nullptr: sizing pass only).
struct Carve {
    unsigned char* base;
    size_t off = 0;
    template <typename T> T* take(size_t n)
    {
        off = (off + kAlign - 1) / kAlign * kAlign;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

struct Buffers {
    double *om64, *wxi64, *weta64;
    void *mon, *disp;
    int2* nodes;
    double *shift, *acc;
    int64_t *n_done, *steps, *paths_run, *next_total, *p_begin, *p_count, *task_off;
    int32_t *node_of, *n_active, *task_counter;
    TaskSlot* slots;
};

size_t carve(Carve& c, Buffers& b, size_t N, size_t M, size_t slots, size_t real_bytes, size_t monb)
{
    b.om64 = c.take<double>(N);
    b.wxi64 = c.take<double>(N);
    b.weta64 = c.take<double>(N);
    b.mon = c.take<unsigned char>(monb);
    b.disp = c.take<unsigned char>(N * 2 * real_bytes);
    b.nodes = c.take<int2>(M);
    b.shift = c.take<double>(2 * M);
    b.acc = c.take<double>(4 * M);
    b.n_done = c.take<int64_t>(M);
    b.steps = c.take<int64_t>(M);
    b.paths_run = c.take<int64_t>(M);
    b.next_total = c.take<int64_t>(M);
    b.p_begin = c.take<int64_t>(M);
    b.p_count = c.take<int64_t>(M);
    b.task_off = c.take<int64_t>(M + 2);
    b.node_of = c.take<int32_t>(M);
    b.n_active = c.take<int32_t>(4);
    b.task_counter = c.take<int32_t>(4);
    b.slots = c.take<TaskSlot>(slots);
    return c.off;
}

// Interface node m -> (i, j) in the canonical order (vertical lines, then horizontal lines
// without the crossings), computed in closed form so no host list is needed.
__global__ void noalloc_nodes_kernel(int nx, int ny, int px, int py, int periodic, int M, int2* nodes)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int sx = (nx - 1) / px, sy = (ny - 1) / py;
    const int nj = periodic ? ny - 1 : ny - 2;   // nodes on one vertical line
    const int nvl = periodic ? px : px - 1;      // vertical lines
    int i, j;
    if (m < nvl * nj) {
        const int line = m / nj;
        i = (periodic ? line : line + 1) * sx;
        j = (periodic ? 0 : 1) + m % nj;
    } else {
        const int k = m - nvl * nj;
        const int per_line = px * (sx - 1);      // nodes of a horizontal line off the crossings
        const int line = k / per_line;
        const int q = k % per_line;
        j = (periodic ? line : line + 1) * sy;
        i = (q / (sx - 1)) * sx + 1 + q % (sx - 1);
    }
    nodes[m] = make_int2(i, j);
}

bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
sdd_status run(const sdd_params* P, const Buffers& b, int M, int acc_mode, int32_t step_index,
               cudaStream_t s)
{
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SDD_ERR_CUDA;
    }
    McParams<T> mp{};
    McProblem<T>& R = mp.prob;
    R.mon = static_cast<const Mon4<T>*>(b.mon);
    R.disp = static_cast<const Disp2<T>*>(b.disp);
    R.nodes = b.nodes;
    R.nx = P->nx; R.ny = P->ny; R.periodic = P->periodic; R.form = P->form; R.K = P->substeps;
    R.bicubic = P->bicubic; R.bb = P->bb_test;
    const T ds = (T)P->dt / (T)P->substeps;
    R.cb = ds / (T)P->tau;
    R.Lx = (T)P->Lx; R.Ly = (T)P->Ly;
    R.key0 = (uint32_t)(P->seed & 0xFFFFFFFFu);
    R.key1 = (uint32_t)(P->seed >> 32);
    philox_round_keys(P->seed, R.rk);
    set_grid_consts(R);
    R.tstep = (uint32_t)step_index;
    R.node_offset = 0;
    mp.shift = b.shift;
    mp.node_of = b.node_of; mp.p_begin = b.p_begin; mp.p_count = b.p_count; mp.task_off = b.task_off;
    mp.n_active = b.n_active; mp.task_counter = b.task_counter; mp.slots = b.slots;

    PlanParams pp{};
    pp.M = M; pp.n_done = b.n_done; pp.next_total = b.next_total; pp.node_of = b.node_of;
    pp.p_begin = b.p_begin; pp.p_count = b.p_count; pp.task_off = b.task_off;
    pp.n_active = b.n_active; pp.task_counter = b.task_counter;
    ReduceParams rp{};
    rp.node_of = b.node_of; rp.p_count = b.p_count; rp.task_off = b.task_off; rp.n_active = b.n_active;
    rp.slots = b.slots; rp.shift = b.shift; rp.acc = b.acc; rp.n_done = b.n_done; rp.steps = b.steps;
    rp.paths_run = b.paths_run; rp.next_total = b.next_total; rp.se_target = 0.0;
    rp.max_paths = P->paths_per_node;

    const int grid = nsm * mc_max_blocks_per_sm<T>(acc_mode, false, false);
    const int64_t rounds = (P->paths_per_node + kMaxChunk - 1) / kMaxChunk;
    if (launch_mc_init(M, P->paths_per_node, P->paths_per_node, b.acc, b.n_done, b.steps, b.paths_run,
                       b.next_total, s) != cudaSuccess)
        return SDD_ERR_CUDA;
    for (int64_t r = 0; r < rounds; ++r) {
        if (launch_plan(pp, s) != cudaSuccess) return SDD_ERR_CUDA;
        if (launch_mc<T>(mp, acc_mode, false, false, grid, s) != cudaSuccess) return SDD_ERR_CUDA;
        if (launch_reduce(rp, M, s) != cudaSuccess) return SDD_ERR_CUDA;
    }
    return SDD_OK;
}

}  // namespace

extern "C" sdd_status sdd_interface_mc_noalloc(const sdd_params* P, const double* x, const double* y,
                                               const double* omega, int32_t step_index, double* est_xy,
                                               double* se_xy, void* stream)
{
    if (!P || !x || !y || !omega || step_index < 0) return SDD_ERR_INVALID_ARG;
    if (P->nx < 3 || P->ny < 3 || P->px < 1 || P->py < 1 || (P->nx - 1) % P->px || (P->ny - 1) % P->py)
        return SDD_ERR_INVALID_ARG;
    if ((P->periodic != 0 && P->periodic != 1) || (P->form != SDD_FORM_DIV && P->form != SDD_FORM_WINSLOW) ||
        P->precision < SDD_FP64 || P->precision > SDD_FP32_KAHAN || (P->bicubic != 0 && P->bicubic != 1) ||
        (P->bb_test != 0 && P->bb_test != 1) || P->substeps < 1 || P->substeps > (1 << 20) ||
        P->iface_stride > 1 || P->iface_stride < 0 || P->moving_boundary != 0)
        return SDD_ERR_INVALID_ARG;
    if (!(P->Lx > 0) || !(P->Ly > 0) || !(P->tau > 0) || !(P->dt > 0) || P->se_target != 0.0 ||
        P->paths_per_node < 2 || P->paths_per_node > (int64_t(1) << 31))
        return SDD_ERR_INVALID_ARG;
    const int sx = (P->nx - 1) / P->px;
    const int64_t nj = P->periodic ? P->ny - 1 : P->ny - 2;
    const int64_t nvl = P->periodic ? P->px : P->px - 1;
    const int64_t nhl = P->periodic ? P->py : P->py - 1;
    const int64_t M = nvl * nj + nhl * (int64_t)P->px * (sx - 1);
    const int64_t N = (int64_t)P->nx * P->ny;
    if (M < 0 || M > (int64_t(1) << 20) || N > (int64_t(1) << 24)) return SDD_ERR_INVALID_ARG;
    if (M > 0 && (!est_xy || !se_xy)) return SDD_ERR_INVALID_ARG;
    const int64_t chunk = P->paths_per_node < kMaxChunk ? P->paths_per_node : kMaxChunk;
    const int64_t slots = M * ((chunk + kPathsPerTask - 1) / kPathsPerTask);
    const bool fp64 = P->precision == SDD_FP64;
    Buffers b{};
    Carve sizing{nullptr};
    if (carve(sizing, b, (size_t)N, (size_t)M, (size_t)slots, fp64 ? 8 : 4, mon_bytes(P->nx, P->ny, fp64)) > kScratchBytes)
        return SDD_ERR_INVALID_ARG;  // larger than the fixed scratch array
    if (!on_device(x) || !on_device(y) || !on_device(omega)) return SDD_ERR_INVALID_ARG;
    if (M == 0) return SDD_OK;  // one Dirichlet subdomain: no interface node, nothing to write
    if (!on_device(est_xy) || !on_device(se_xy)) return SDD_ERR_INVALID_ARG;
    void* base = nullptr;
    const sdd_status st = scratch_for_current_device(&base);
    if (st != SDD_OK) return st;
    Carve c{static_cast<unsigned char*>(base)};
    carve(c, b, (size_t)N, (size_t)M, (size_t)slots, fp64 ? 8 : 4, mon_bytes(P->nx, P->ny, fp64));
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    noalloc_nodes_kernel<<<(int)((M + 255) / 256), 256, 0, s>>>(P->nx, P->ny, P->px, P->py, P->periodic,
                                                                (int)M, b.nodes);
    if (cudaGetLastError() != cudaSuccess) return SDD_ERR_CUDA;
    PrepParams pr{};
    pr.nx = P->nx; pr.ny = P->ny; pr.periodic = P->periodic; pr.kind = SDD_MONITOR_NODAL; pr.n_params = 0;
    pr.precision = P->precision; pr.Lx = P->Lx; pr.Ly = P->Ly; pr.t = P->t0 + step_index * P->dt;
    pr.x = x; pr.y = y; pr.omega_in = omega;
    pr.om64 = b.om64; pr.wxi64 = b.wxi64; pr.weta64 = b.weta64; pr.mon = b.mon; pr.disp = b.disp;
    if (launch_prep(pr, s) != cudaSuccess) return SDD_ERR_CUDA;
    if (launch_shift(b.nodes, (int)M, P->nx, x, y, b.shift, s) != cudaSuccess) return SDD_ERR_CUDA;
    const int acc_mode = P->precision == SDD_FP32_KAHAN ? kAccKahan32 : kAcc64;
    const sdd_status r = fp64 ? run<double>(P, b, (int)M, acc_mode, step_index, s)
                              : run<float>(P, b, (int)M, acc_mode, step_index, s);
    if (r != SDD_OK) return r;
    if (launch_output((int)M, b.acc, b.n_done, b.shift, est_xy, se_xy, s) != cudaSuccess) return SDD_ERR_CUDA;
    return SDD_OK;
}
