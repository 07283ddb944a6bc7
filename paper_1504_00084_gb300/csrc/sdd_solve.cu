// Backward-Euler subdomain solves of the SDD mesh generator (Sec. 3.5), sm_103a.
//
// Every subdomain is an independent Dirichlet problem (interface estimates and physical
// boundary on its rim).  For interior node P with neighbours E, W, N, S the step solves
//   d_P x_P + sum_nb c_nb (x_P - x_nb) = d_P x^n_P,
//   c_E = (dt/tau) (omega_P + omega_E)/2 / h_xi^2  (likewise W, N, S with h_eta),
//   d_P = 1 (tau x_t = div(omega grad x))  or  omega_P (the paper's Eq. 4 form),
// a symmetric positive-definite system, for both mesh components at once.
//
// One CTA of 512 threads per subdomain, two per SM, or a cluster of CTAs for a large subdomain
// (solve_item).  Outer loop in FP64: residual b - A x of the current iterate (rims
// included), stop when ||r||_2 <= rtol ||b||_2 for both components.  Inner solve A e = r by
// conjugate gradients in the inner precision (FP32 for the FP32 modes, FP64 otherwise),
// preconditioned by one symmetric multigrid V-cycle, then x += e (iterative refinement).
//
// Multigrid: the subdomain's interior (n x m nodes) coarsens to the nodes of odd index,
// (n-1)/2 of them for odd n and n/2 for even n (the last coarse node then lies one fine spacing
// from the rim), for as long as both sizes stay >= 3.  Coarse face
// coefficients are a quarter of the series combination 2ab/(a+b) of the two fine faces a
// coarse face spans (the operator rediscretised at twice the spacing); the identity term is
// injected.  Red-black Gauss-Seidel smoothing (red-black before, black-red after: a symmetric
// cycle), full-weighting restriction, bilinear prolongation, symmetric Gauss-Seidel sweeps on
// the coarsest level; zero rims on every level (the cycle acts on residual equations).  Inner vectors live in full-grid arrays whose rim
// entries stay zero, so A p needs no rim special cases.  All reductions are fixed-order
// block trees: the solve is deterministic.
#include <cooperative_groups.h>
#include <math.h>

#include "sdd_internal.cuh"

namespace sdd {

namespace {

// 512 threads per CTA, two CTAs per SM (64 registers each): a subdomain gets 16 warps, and an SM
// keeps two subdomains' passes in flight; a large subdomain gets a cluster of kCoopWidth CTAs.
// Measured on the 64-problem mix: 10.9-12.4 ms per batched solve, against 15.4-17.3 ms with one
// 1024-thread CTA per SM (and clusters of 2) and 12.1-13.7 ms with 256-thread CTAs.
constexpr int kSolveThreads = 512;
constexpr int kSolveMinBlocks = 1024 / kSolveThreads;
constexpr int kMaxOuter = 12;
constexpr int kCoarseSweeps = 4;  // symmetric Gauss-Seidel sweeps on the coarsest level
constexpr unsigned kFull = 0xffffffffu;

template <typename TI> struct Pair {
    TI x, y;
};

#ifndef SDD_SOLVE_ILP
#define SDD_SOLVE_ILP 1   // nodes per lane whose loads are issued together in a half-sweep
#endif
constexpr int kIlp = 1;
constexpr int kIlpSweep = SDD_SOLVE_ILP;

// The CTAs that solve one subdomain together: one CTA (CW = 1), or the CW CTAs of a thread-block
// cluster (a large subdomain).  Rows, loops and reductions are spread over all of the team's
// threads; sync() is the CTA barrier or the cluster barrier, which also orders the team's global
// memory writes before the reads that follow it.
template <int CW> struct Team {
    int rank;  // rank of this CTA in the team (0 when CW = 1)
    __device__ __forceinline__ int tid() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ __forceinline__ int nthreads() const { return CW * (int)blockDim.x; }
    __device__ __forceinline__ int warp() const { return rank * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); }
    __device__ __forceinline__ int nwarps() const { return CW * (int)(blockDim.x >> 5); }
    __device__ __forceinline__ void sync() const
    {
        if constexpr (CW == 1) __syncthreads();
        else cooperative_groups::this_cluster().sync();
    }
};

// Visits the nodes (i, j) of an nx x ny row-major array.  Warp w of the team takes rows w, w + W,
// ...; in a row, lane l takes columns c0 + s (l + 32 u) for u < U, with s = 1 and c0 = 0
// (colour < 0), or s = 2 and c0 = (j + colour) & 1 (the nodes with (i + j) % 2 == colour).
// value(i, j) computes a node's result from loads only and put(i, j, v) stores it: a lane issues
// the loads of its U nodes before any store, so U nodes' memory requests are in flight together,
// and no index is divided.
template <int U, int CW, typename Value, typename Put>
__device__ __forceinline__ void for_rows(const Team<CW>& tm, int nx, int ny, int colour, Value value, Put put)
{
    using V = decltype(value(0, 0));
    const int lane = threadIdx.x & 31, W = tm.nwarps();
    const int st = colour < 0 ? 1 : 2;
    for (int j = tm.warp(); j < ny; j += W) {
        const int c0 = colour < 0 ? 0 : ((j + colour) & 1);
        for (int b = c0 + st * lane; b < nx; b += st * 32 * U) {
            V v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (b + st * 32 * u < nx) v[u] = value(b + st * 32 * u, j);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (b + st * 32 * u < nx) put(b + st * 32 * u, j, v[u]);
        }
    }
}

// Sum of NV doubles over the team; every thread receives the totals.  Within a CTA a fixed
// warp tree; across the CTAs of a cluster the CTA totals in rank order (read from each CTA's
// shared memory), so every thread of the team gets the same bits.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh);

template <int CW, int NV>
__device__ __forceinline__ void team_sum(const Team<CW>& tm, double (&v)[NV], double* sh)
{
    if constexpr (CW == 1) {
        block_sum<NV>(v, sh);
    } else {
        namespace cg = cooperative_groups;
        block_sum<NV>(v, sh);                  // this CTA's totals, also left in sh[32 NV + 32 k]
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();                             // every CTA's totals are in place
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int r = 0; r < CW; ++r) t += *cl.map_shared_rank(sh + 32 * NV + 32 * k, r);
            v[k] = t;
        }
        cl.sync();                             // nobody overwrites sh before all have read it
    }
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(kFull, t, off);
            if (lane == 0) sh[k * 32 + 32 * NV] = t;  // slot after the per-warp table
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = sh[k * 32 + 32 * NV];
    __syncthreads();
}

__device__ __forceinline__ void faces_body(const SolveParams& P, int inner_fp64, int blk, int nb)
{
    const int nx = P.nx, ny = P.ny;
    const double hx2 = (double)(nx - 1) * (double)(nx - 1);
    const double hy2 = (double)(ny - 1) * (double)(ny - 1);
    const long n = (long)nx * ny;
    for (long id = blk * (long)blockDim.x + threadIdx.x; id < n; id += (long)nb * blockDim.x) {
        const int i = (int)(id % nx), j = (int)(id / nx);
        const double w = P.om64[id];
        double e = 0.0, no = 0.0;
        if (i < nx - 1) e = __dmul_rn(P.r, __dmul_rn(__dmul_rn(0.5, __dadd_rn(w, P.om64[id + 1])), hx2));
        if (j < ny - 1) no = __dmul_rn(P.r, __dmul_rn(__dmul_rn(0.5, __dadd_rn(w, P.om64[id + nx])), hy2));
        P.ce64[id] = e;
        P.cn64[id] = no;
        if (inner_fp64) {
            static_cast<double*>(P.ce)[id] = e;
            static_cast<double*>(P.cn)[id] = no;
        } else {
            static_cast<float*>(P.ce)[id] = (float)e;
            static_cast<float*>(P.cn)[id] = (float)no;
        }
    }
}

__global__ void faces_kernel(const SolveParams P, int inner_fp64) { faces_body(P, inner_fp64, blockIdx.x, gridDim.x); }

// Face coefficients of every problem of a batch in one launch (problem i: blocks blk_off[i] ..).
__global__ void faces_batch_kernel(const SolveParams* probs, const int32_t* blk_off, int n, int inner_fp64)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    faces_body(probs[lo], inner_fp64, blockIdx.x - blk_off[lo], blk_off[lo + 1] - blk_off[lo]);
}


// ------------------------------------------------------------------------------------------
// Multigrid hierarchy of one subdomain: compact per-level arrays in the subdomain's workspace.
// ------------------------------------------------------------------------------------------
template <typename TI> struct MgLevel {
    int nx, ny;
    Pair<TI>* x;   // correction
    Pair<TI>* b;   // right-hand side
    Pair<TI>* t;   // residual
    TI* ce;        // faces along xi: (nx + 1) per row, face f between nodes f-1 and f
    TI* cn;        // faces along eta: (ny + 1) rows of nx
    TI* d;         // identity term
};

template <typename TI>
__device__ __forceinline__ MgLevel<TI> mg_level(void* base, int nx0, int ny0, int l)
{
    char* ptr = static_cast<char*>(base);
    int nx = nx0, ny = ny0;
    for (int k = 0;; ++k) {
        MgLevel<TI> L;
        L.nx = nx; L.ny = ny;
        const size_t nn = (size_t)nx * ny;
        L.x = reinterpret_cast<Pair<TI>*>(ptr); ptr += mg_align(nn * sizeof(Pair<TI>));
        L.b = reinterpret_cast<Pair<TI>*>(ptr); ptr += mg_align(nn * sizeof(Pair<TI>));
        L.t = reinterpret_cast<Pair<TI>*>(ptr); ptr += mg_align(nn * sizeof(Pair<TI>));
        L.ce = reinterpret_cast<TI*>(ptr); ptr += mg_align((size_t)(nx + 1) * ny * sizeof(TI));
        L.cn = reinterpret_cast<TI*>(ptr); ptr += mg_align((size_t)nx * (ny + 1) * sizeof(TI));
        L.d = reinterpret_cast<TI*>(ptr); ptr += mg_align(nn * sizeof(TI));
        if (k == l) return L;
        nx = mg_coarse(nx);
        ny = mg_coarse(ny);
    }
}

template <typename TI>
__device__ __forceinline__ TI mg_diag(const MgLevel<TI>& L, int i, int j)
{
    return L.d[j * L.nx + i] + L.ce[j * (L.nx + 1) + i] + L.ce[j * (L.nx + 1) + i + 1] +
           L.cn[j * L.nx + i] + L.cn[(j + 1) * L.nx + i];
}

// sum over the four neighbours of c_nb * x_nb (zero outside the level's interior)
template <typename TI>
__device__ __forceinline__ Pair<TI> mg_offdiag(const MgLevel<TI>& L, int i, int j)
{
    const int nx = L.nx, ny = L.ny, id = j * nx + i;
    Pair<TI> s{(TI)0, (TI)0};
    if (i > 0) { const TI c = L.ce[j * (nx + 1) + i]; s.x += c * L.x[id - 1].x; s.y += c * L.x[id - 1].y; }
    if (i < nx - 1) { const TI c = L.ce[j * (nx + 1) + i + 1]; s.x += c * L.x[id + 1].x; s.y += c * L.x[id + 1].y; }
    if (j > 0) { const TI c = L.cn[j * nx + i]; s.x += c * L.x[id - nx].x; s.y += c * L.x[id - nx].y; }
    if (j < ny - 1) { const TI c = L.cn[(j + 1) * nx + i]; s.x += c * L.x[id + nx].x; s.y += c * L.x[id + nx].y; }
    return s;
}

// one Gauss-Seidel half-sweep over the nodes of one colour ((i + j) % 2 == colour)
template <typename TI, int CW>
__device__ __forceinline__ void mg_half_sweep(const Team<CW>& tm, const MgLevel<TI>& L, int colour)
{
    for_rows<kIlpSweep>(tm, 
        L.nx, L.ny, colour,
        [&](int i, int j) {
            const Pair<TI> o = mg_offdiag(L, i, j);
            const TI dg = mg_diag(L, i, j);
            const Pair<TI> bb = L.b[j * L.nx + i];
            return Pair<TI>{(bb.x + o.x) / dg, (bb.y + o.y) / dg};
        },
        [&](int i, int j, const Pair<TI>& v) { L.x[j * L.nx + i] = v; });
    tm.sync();
}

// The first half-sweep of a level from a zero initial guess, in one pass: nodes of colour 0 take
// b / diag (their neighbours are still zero), nodes of colour 1 are zeroed.
template <typename TI, int CW>
__device__ __forceinline__ void mg_first_sweep(const Team<CW>& tm, const MgLevel<TI>& L)
{
    for_rows<kIlpSweep>(tm,
        L.nx, L.ny, -1,
        [&](int i, int j) {
            if ((i + j) & 1) return Pair<TI>{(TI)0, (TI)0};
            const TI dg = mg_diag(L, i, j);
            const Pair<TI> bb = L.b[j * L.nx + i];
            return Pair<TI>{bb.x / dg, bb.y / dg};
        },
        [&](int i, int j, const Pair<TI>& v) { L.x[j * L.nx + i] = v; });
    tm.sync();
}

template <typename TI, int CW>
__device__ __forceinline__ void mg_zero(const Team<CW>& tm, const MgLevel<TI>& L)
{
    for (int k = tm.tid(); k < L.nx * L.ny; k += tm.nthreads()) L.x[k] = Pair<TI>{(TI)0, (TI)0};
    tm.sync();
}

// b_{l+1} = full weighting of the residual t_l = b_l - A_l x_l
template <typename TI, int CW>
__device__ __forceinline__ void mg_restrict(const Team<CW>& tm, const MgLevel<TI>& F, const MgLevel<TI>& C)
{
    for_rows<kIlp>(tm, 
        F.nx, F.ny, -1,
        [&](int i, int j) {
            const int k = j * F.nx + i;
            const Pair<TI> o = mg_offdiag(F, i, j);
            const TI dg = mg_diag(F, i, j);
            const Pair<TI> xv = F.x[k], bv = F.b[k];
            return Pair<TI>{bv.x - (dg * xv.x - o.x), bv.y - (dg * xv.y - o.y)};
        },
        [&](int i, int j, const Pair<TI>& v) { F.t[j * F.nx + i] = v; });
    tm.sync();
    for_rows<kIlp>(tm, 
        C.nx, C.ny, -1,
        [&](int I, int J) {
            const int i = 2 * I + 1, j = 2 * J + 1;
            Pair<TI> acc{(TI)0, (TI)0};
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
                for (int di = -1; di <= 1; ++di) {
                    // an even fine size puts the last coarse node's outer neighbours on the rim,
                    // whose residual is zero
                    if (i + di >= F.nx || j + dj >= F.ny) continue;
                    const TI w = (TI)((di == 0 ? 2 : 1) * (dj == 0 ? 2 : 1)) * (TI)0.0625;
                    const Pair<TI> tv = F.t[(j + dj) * F.nx + (i + di)];
                    acc.x += w * tv.x;
                    acc.y += w * tv.y;
                }
            return acc;
        },
        [&](int I, int J, const Pair<TI>& v) { C.b[J * C.nx + I] = v; });
    tm.sync();
}

// x_l += bilinear interpolation of x_{l+1} (coarse rims are zero)
template <typename TI, int CW>
__device__ __forceinline__ void mg_prolong(const Team<CW>& tm, const MgLevel<TI>& F, const MgLevel<TI>& C)
{
    for_rows<kIlp>(tm, F.nx, F.ny, -1, [&](int i, int j) {
        // coarse neighbours: odd fine index 2I+1 -> I; even fine index 2I -> I-1 and I
        const int Ia = (i & 1) ? (i - 1) / 2 : i / 2 - 1, Ib = (i & 1) ? Ia : i / 2;
        const int Ja = (j & 1) ? (j - 1) / 2 : j / 2 - 1, Jb = (j & 1) ? Ja : j / 2;
        const TI wi = (i & 1) ? (TI)1 : (TI)0.5, wj = (j & 1) ? (TI)1 : (TI)0.5;
        Pair<TI> s{(TI)0, (TI)0};
        const int Is[2] = {Ia, Ib}, Js[2] = {Ja, Jb};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (((i & 1) && a == 1) || ((j & 1) && c == 1)) continue;
                const int I = Is[a], J = Js[c];
                if (I < 0 || I >= C.nx || J < 0 || J >= C.ny) continue;
                const Pair<TI> v = C.x[J * C.nx + I];
                s.x += wi * wj * v.x;
                s.y += wi * wj * v.y;
            }
        const Pair<TI> f = F.x[j * F.nx + i];
        return Pair<TI>{f.x + s.x, f.y + s.y};
    }, [&](int i, int j, const Pair<TI>& v) { F.x[j * F.nx + i] = v; });
    tm.sync();
}

// Coefficients of every level from the fine face coefficients of the subdomain.
template <typename TI, int CW>
__device__ void mg_setup(const Team<CW>& tm, const SolveParams& P, int i0, int j0, int nx0, int ny0, int levels)
{
    const TI* ce = static_cast<const TI*>(P.ce);
    const TI* cn = static_cast<const TI*>(P.cn);
    const int nx = P.nx;
    const MgLevel<TI> L0 = mg_level<TI>(P.mg, nx0, ny0, 0);
    for (int k = tm.tid(); k < (nx0 + 1) * ny0; k += tm.nthreads()) {
        const int f = k % (nx0 + 1), j = k / (nx0 + 1);
        L0.ce[k] = ce[(long)(j0 + 1 + j) * nx + (i0 + f)];
    }
    for (int k = tm.tid(); k < nx0 * (ny0 + 1); k += tm.nthreads()) {
        const int i = k % nx0, g = k / nx0;
        L0.cn[k] = cn[(long)(j0 + g) * nx + (i0 + 1 + i)];
    }
    for (int k = tm.tid(); k < nx0 * ny0; k += tm.nthreads()) {
        const int i = k % nx0, j = k / nx0;
        L0.d[k] = P.form == 0 ? (TI)1 : (TI)P.om64[(long)(j0 + 1 + j) * nx + (i0 + 1 + i)];
    }
    tm.sync();
    for (int l = 0; l + 1 < levels; ++l) {
        const MgLevel<TI> F = mg_level<TI>(P.mg, nx0, ny0, l), C = mg_level<TI>(P.mg, nx0, ny0, l + 1);
        // a coarse face spans two fine faces (a quarter of their series combination), except the
        // face to the rim after an even fine size, which spans one fine face at one fine spacing
        // from the rim: half of it
        for (int k = tm.tid(); k < (C.nx + 1) * C.ny; k += tm.nthreads()) {
            const int f = k % (C.nx + 1), J = k / (C.nx + 1);
            const TI a = F.ce[(2 * J + 1) * (F.nx + 1) + 2 * f];
            if (2 * f + 1 > F.nx) { C.ce[k] = (TI)0.5 * a; continue; }
            const TI b = F.ce[(2 * J + 1) * (F.nx + 1) + 2 * f + 1];
            C.ce[k] = (TI)0.5 * a * b / (a + b);
        }
        for (int k = tm.tid(); k < C.nx * (C.ny + 1); k += tm.nthreads()) {
            const int I = k % C.nx, g = k / C.nx;
            const TI a = F.cn[(2 * g) * F.nx + 2 * I + 1];
            if (2 * g + 1 > F.ny) { C.cn[k] = (TI)0.5 * a; continue; }
            const TI b = F.cn[(2 * g + 1) * F.nx + 2 * I + 1];
            C.cn[k] = (TI)0.5 * a * b / (a + b);
        }
        for (int k = tm.tid(); k < C.nx * C.ny; k += tm.nthreads()) {
            const int I = k % C.nx, J = k / C.nx;
            C.d[k] = F.d[(2 * J + 1) * F.nx + 2 * I + 1];
        }
        tm.sync();
    }
}

// x_0 = V-cycle(b_0): one symmetric multigrid cycle.
template <typename TI, int CW>
__device__ __noinline__ void mg_vcycle(const Team<CW> tm, void* base, int nx0, int ny0, int levels)
{
    for (int l = 0; l + 1 < levels; ++l) {
        const MgLevel<TI> F = mg_level<TI>(base, nx0, ny0, l);
        mg_first_sweep(tm, F);
        mg_half_sweep(tm, F, 1);
        mg_restrict(tm, F, mg_level<TI>(base, nx0, ny0, l + 1));
    }
    const MgLevel<TI> Lc = mg_level<TI>(base, nx0, ny0, levels - 1);
    if (Lc.nx * Lc.ny == 1) {
        // one node, no neighbours: the first half-sweep solves it exactly (b / diag), and every
        // further sweep would recompute the same bits
        mg_first_sweep(tm, Lc);
    } else {
        for (int s = 0; s < kCoarseSweeps; ++s) {
            if (s == 0) mg_first_sweep(tm, Lc);
            else mg_half_sweep(tm, Lc, 0);
            mg_half_sweep(tm, Lc, 1);
            mg_half_sweep(tm, Lc, 1);
            mg_half_sweep(tm, Lc, 0);
        }
    }
    for (int l = levels - 2; l >= 0; --l) {
        const MgLevel<TI> F = mg_level<TI>(base, nx0, ny0, l);
        mg_prolong(tm, F, mg_level<TI>(base, nx0, ny0, l + 1));
        mg_half_sweep(tm, F, 1);
        mg_half_sweep(tm, F, 0);
    }
}

// Largest value of v over the block; every thread receives it.
__device__ __forceinline__ double block_max(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, off));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t = fmax(t, __shfl_xor_sync(kFull, t, off));
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// Forward Euler (the paper's local solver, Sec. 3.5) for subdomain `sub`, in FP64: S substeps of
//   x_P <- x_P + (1 / (S d_P)) sum_nb c_nb (x_nb - x_P),   S = ceil(max_P sum_nb c_nb / d_P),
// so every substep is a convex combination (discrete maximum principle); a rim neighbour takes
// x^n + (m / S)(x^{n+1} - x^n) at substep m.  Two full-grid FP64 pair buffers in P.vec hold the
// interior iterates (the inner-vector storage, unused by this scheme).
__device__ void fe_body(const SolveParams& P, int sub, double* sh)
{
    const int nx = P.nx, ny = P.ny;
    const int I = sub % P.px, J = sub / P.px;
    const int i0 = split_line(I, nx, P.px), i1 = split_line(I + 1, nx, P.px);
    const int j0 = split_line(J, ny, P.py), j1 = split_line(J + 1, ny, P.py);
    const int ni = i1 - i0 - 1, nj = j1 - j0 - 1;
    const int nint = ni * nj;
    const long N = (long)nx * ny;
    double2* A = static_cast<double2*>(P.vec);
    double2* B = A + N;
    auto node = [&](int t) -> long { return (long)(j0 + 1 + t / ni) * nx + (i0 + 1 + t % ni); };
    auto dP = [&](long id) -> double { return P.form == 0 ? 1.0 : P.om64[id]; };
    double cmax = 0.0;
    for (int t = threadIdx.x; t < nint; t += blockDim.x) {
        const long id = node(t);
        const double c = __dadd_rn(__dadd_rn(__dadd_rn(P.ce64[id], P.ce64[id - 1]), P.cn64[id]), P.cn64[id - nx]);
        cmax = fmax(cmax, __ddiv_rn(c, dP(id)));
    }
    cmax = block_max(cmax, sh);
    const double Sd = ceil(cmax) < 1.0 ? 1.0 : ceil(cmax);
    if (!(Sd <= (double)P.fe_max_substeps)) {
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const long id = node(t);
            P.xnew[id] = P.xcur[id];
            P.ynew[id] = P.ycur[id];
        }
        if (threadIdx.x == 0) {
            P.stat_iters[sub] = 0; P.stat_outer[sub] = 0; P.stat_ok[sub] = 0; P.stat_res[sub] = 0.0;
        }
        return;
    }
    const int S = (int)Sd;
    for (int t = threadIdx.x; t < nint; t += blockDim.x) {
        const long id = node(t);
        A[id] = make_double2(P.xcur[id], P.ycur[id]);
    }
    __syncthreads();
    for (int m = 0; m < S; ++m) {
        const double f = __ddiv_rn((double)m, Sd);
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const long id = node(t);
            const int i = (int)(id % nx), j = (int)(id / nx);
            auto val = [&](long nb, bool rim) -> double2 {
                if (!rim) return A[nb];
                const double px = P.xcur[nb], py = P.ycur[nb];
                return make_double2(__dadd_rn(px, __dmul_rn(f, __dsub_rn(P.xnew[nb], px))),
                                    __dadd_rn(py, __dmul_rn(f, __dsub_rn(P.ynew[nb], py))));
            };
            const double2 c = A[id];
            const double2 vE = val(id + 1, i + 1 == i1), vW = val(id - 1, i - 1 == i0);
            const double2 vN = val(id + nx, j + 1 == j1), vS = val(id - nx, j - 1 == j0);
            const double cE = P.ce64[id], cW = P.ce64[id - 1], cN = P.cn64[id], cS = P.cn64[id - nx];
            const double sx = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(cE, __dsub_rn(vE.x, c.x)), __dmul_rn(cW, __dsub_rn(vW.x, c.x))),
                                                  __dmul_rn(cN, __dsub_rn(vN.x, c.x))), __dmul_rn(cS, __dsub_rn(vS.x, c.x)));
            const double sy = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(cE, __dsub_rn(vE.y, c.y)), __dmul_rn(cW, __dsub_rn(vW.y, c.y))),
                                                  __dmul_rn(cN, __dsub_rn(vN.y, c.y))), __dmul_rn(cS, __dsub_rn(vS.y, c.y)));
            const double den = __dmul_rn(Sd, dP(id));
            B[id] = make_double2(__dadd_rn(c.x, __ddiv_rn(sx, den)), __dadd_rn(c.y, __ddiv_rn(sy, den)));
        }
        __syncthreads();
        double2* tmp = A;
        A = B;
        B = tmp;
    }
    for (int t = threadIdx.x; t < nint; t += blockDim.x) {
        const long id = node(t);
        P.xnew[id] = A[id].x;
        P.ynew[id] = A[id].y;
    }
    if (threadIdx.x == 0) {
        P.stat_iters[sub] = S; P.stat_outer[sub] = 0; P.stat_ok[sub] = 1; P.stat_res[sub] = 0.0;
    }
}

// Subdomain `sub` of the problem described by P, solved by the calling CTA.
template <typename TI, int CW>
__device__ __forceinline__ void solve_body(const Team<CW>& tm, const SolveParams& P, int sub, double* sh)
{
    const int nx = P.nx, ny = P.ny;
    const int I = sub % P.px, J = sub / P.px;
    const int i0 = split_line(I, nx, P.px), i1 = split_line(I + 1, nx, P.px);
    const int j0 = split_line(J, ny, P.py), j1 = split_line(J + 1, ny, P.py);
    const int ni = i1 - i0 - 1, nj = j1 - j0 - 1;
    const int nint = ni * nj;
    const long N = (long)nx * ny;
    Pair<TI>* e = static_cast<Pair<TI>*>(P.vec);
    Pair<TI>* r = e + N;
    Pair<TI>* p = e + 2 * N;
    Pair<TI>* q = e + 3 * N;
    const TI* ce = static_cast<const TI*>(P.ce);
    const TI* cn = static_cast<const TI*>(P.cn);

    // interior node (ii, jj) of the subdomain: full-grid index; its compact index is jj * ni + ii
    auto gid = [&](int ii, int jj) -> long { return (long)(j0 + 1 + jj) * nx + (i0 + 1 + ii); };
    auto dP = [&](long id) -> double { return P.form == 0 ? 1.0 : P.om64[id]; };

    // initial guess: the previous mesh
    for_rows<kIlp>(tm, 
        ni, nj, -1, [&](int ii, int jj) { const long id = gid(ii, jj); return Pair<double>{P.xcur[id], P.ycur[id]}; },
        [&](int ii, int jj, const Pair<double>& v) { const long id = gid(ii, jj); P.xnew[id] = v.x; P.ynew[id] = v.y; });
    // ||b||: b = d x^n + rim terms (rim values are the new Dirichlet data, not written here)
    double bn[2] = {0.0, 0.0};
    for_rows<kIlp>(tm, 
        ni, nj, -1,
        [&](int ii, int jj) {
            const long id = gid(ii, jj);
            const int i = i0 + 1 + ii, j = j0 + 1 + jj;
            const double d = dP(id);
            double bx = d * P.xcur[id], by = d * P.ycur[id];
            if (i - 1 == i0) { bx += P.ce64[id - 1] * P.xnew[id - 1]; by += P.ce64[id - 1] * P.ynew[id - 1]; }
            if (i + 1 == i1) { bx += P.ce64[id] * P.xnew[id + 1]; by += P.ce64[id] * P.ynew[id + 1]; }
            if (j - 1 == j0) { bx += P.cn64[id - nx] * P.xnew[id - nx]; by += P.cn64[id - nx] * P.ynew[id - nx]; }
            if (j + 1 == j1) { bx += P.cn64[id] * P.xnew[id + nx]; by += P.cn64[id] * P.ynew[id + nx]; }
            return Pair<double>{bx, by};
        },
        [&](int, int, const Pair<double>& v) { bn[0] += v.x * v.x; bn[1] += v.y * v.y; });
    tm.sync();
    team_sum<CW, 2>(tm, bn, sh);

    // multigrid hierarchy of this subdomain
    void* mgbase = static_cast<char*>(P.mg) + (size_t)sub * P.mg_stride;
    SolveParams Pm = P;
    Pm.mg = mgbase;
    const int levels = mg_levels(ni, nj);
    if (nint > 0) mg_setup<TI>(tm, Pm, i0, j0, ni, nj, levels);
    const MgLevel<TI> L0 = mg_level<TI>(mgbase, ni, nj, 0);
    // z = V-cycle(r) into L0.x (interior-compact), from the full-grid residual r
    // (the passes that write r also write it into L0.b, the right-hand side of the cycle)
    auto precondition = [&]() { mg_vcycle<TI>(tm, mgbase, ni, nj, levels); };

    const bool fp64_inner = sizeof(TI) == 8;
    int iters = 0, outer = 0, ok = 0;
    double rel = 0.0;
    for (outer = 0; outer < kMaxOuter; ++outer) {
        // FP64 residual of the current iterate
        double rn[2] = {0.0, 0.0};
        for_rows<kIlp>(tm, 
            ni, nj, -1,
            [&](int ii, int jj) {
                const long id = gid(ii, jj);
                const double cE = P.ce64[id], cW = P.ce64[id - 1], cN = P.cn64[id], cS = P.cn64[id - nx];
                const double d = dP(id);
                const double diag = d + cE + cW + cN + cS;
                const double ax = diag * P.xnew[id] - cE * P.xnew[id + 1] - cW * P.xnew[id - 1] -
                                  cN * P.xnew[id + nx] - cS * P.xnew[id - nx];
                const double ay = diag * P.ynew[id] - cE * P.ynew[id + 1] - cW * P.ynew[id - 1] -
                                  cN * P.ynew[id + nx] - cS * P.ynew[id - nx];
                return Pair<double>{d * P.xcur[id] - ax, d * P.ycur[id] - ay};
            },
            [&](int ii, int jj, const Pair<double>& v) {
                const Pair<TI> rv{(TI)v.x, (TI)v.y};
                r[gid(ii, jj)] = rv;
                L0.b[jj * ni + ii] = rv;
                rn[0] += v.x * v.x;
                rn[1] += v.y * v.y;
            });
        tm.sync();
        team_sum<CW, 2>(tm, rn, sh);
        const double relx = bn[0] > 0 ? sqrt(rn[0] / bn[0]) : sqrt(rn[0]);
        const double rely = bn[1] > 0 ? sqrt(rn[1] / bn[1]) : sqrt(rn[1]);
        rel = relx > rely ? relx : rely;
        if (rel <= P.rtol) {
            ok = 1;
            break;
        }
        if (iters >= P.max_iter) break;
        // inner relative tolerance: straight to the target in FP64, 1e-5 per sweep in FP32 (two
        // sweeps reach 1e-10 from the previous mesh; 1e-4 took three, 1e-6 meets FP32 stagnation)
        double tol_rel[2];
        for (int c = 0; c < 2; ++c) {
            const double cur = c == 0 ? relx : rely;
            double t = fp64_inner ? 0.5 * P.rtol / (cur > 0 ? cur : 1.0) : 1e-5;
            if (fp64_inner && t < 1e-14) t = 1e-14;
            if (t > 0.5) t = 0.5;
            tol_rel[c] = t;
        }
        // CG start: e = 0, p = z = M^-1 r (one V-cycle)
        precondition();
        double rz[2] = {0.0, 0.0}, rr0[2] = {0.0, 0.0};
        for_rows<kIlp>(tm, 
            ni, nj, -1, [&](int ii, int jj) { return Pair<Pair<TI>>{r[gid(ii, jj)], L0.x[jj * ni + ii]}; },
            [&](int ii, int jj, const Pair<Pair<TI>>& v) {
                const long id = gid(ii, jj);
                const Pair<TI> rv = v.x, z = v.y;
                e[id] = Pair<TI>{(TI)0, (TI)0};
                p[id] = z;
                rz[0] += (double)rv.x * (double)z.x;
                rz[1] += (double)rv.y * (double)z.y;
                rr0[0] += (double)rv.x * (double)rv.x;
                rr0[1] += (double)rv.y * (double)rv.y;
            });
        tm.sync();
        {
            double v[4] = {rz[0], rz[1], rr0[0], rr0[1]};
            team_sum<CW, 4>(tm, v, sh);
            rz[0] = v[0]; rz[1] = v[1]; rr0[0] = v[2]; rr0[1] = v[3];
        }
        bool done_c[2] = {rr0[0] == 0.0, rr0[1] == 0.0};
        while (iters < P.max_iter && !(done_c[0] && done_c[1])) {
            ++iters;
            double pq[2] = {0.0, 0.0};
            for_rows<kIlp>(tm, 
                ni, nj, -1,
                [&](int ii, int jj) {
                    const long id = gid(ii, jj);
                    const TI cE = ce[id], cW = ce[id - 1], cN = cn[id], cS = cn[id - nx];
                    const TI diag = (TI)dP(id) + cE + cW + cN + cS;
                    const Pair<TI> pc = p[id], pe = p[id + 1], pw = p[id - 1], pn = p[id + nx], ps = p[id - nx];
                    return Pair<Pair<TI>>{pc, Pair<TI>{diag * pc.x - cE * pe.x - cW * pw.x - cN * pn.x - cS * ps.x,
                                                       diag * pc.y - cE * pe.y - cW * pw.y - cN * pn.y - cS * ps.y}};
                },
                [&](int ii, int jj, const Pair<Pair<TI>>& v) {
                    q[gid(ii, jj)] = v.y;
                    pq[0] += (double)v.x.x * (double)v.y.x;
                    pq[1] += (double)v.x.y * (double)v.y.y;
                });
            tm.sync();
            team_sum<CW, 2>(tm, pq, sh);
            const TI ax = (!done_c[0] && pq[0] > 0) ? (TI)(rz[0] / pq[0]) : (TI)0;
            const TI ay = (!done_c[1] && pq[1] > 0) ? (TI)(rz[1] / pq[1]) : (TI)0;
            double v[4] = {0.0, 0.0, 0.0, 0.0};  // r.z (x, y), r.r (x, y)
            for_rows<kIlp>(tm, 
                ni, nj, -1,
                [&](int ii, int jj) {
                    const long id = gid(ii, jj);
                    const Pair<TI> pc = p[id], qv = q[id];
                    Pair<TI> ev = e[id], rv = r[id];
                    ev.x += ax * pc.x; ev.y += ay * pc.y;
                    rv.x -= ax * qv.x; rv.y -= ay * qv.y;
                    return Pair<Pair<TI>>{ev, rv};
                },
                [&](int ii, int jj, const Pair<Pair<TI>>& v) {
                    const long id = gid(ii, jj);
                    e[id] = v.x;
                    r[id] = v.y;
                    L0.b[jj * ni + ii] = v.y;
                });
            tm.sync();
            precondition();
            for_rows<kIlp>(tm, 
                ni, nj, -1, [&](int ii, int jj) { return Pair<Pair<TI>>{r[gid(ii, jj)], L0.x[jj * ni + ii]}; },
                [&](int, int, const Pair<Pair<TI>>& w) {
                    const Pair<TI> rv = w.x, z = w.y;
                    v[0] += (double)rv.x * (double)z.x;
                    v[1] += (double)rv.y * (double)z.y;
                    v[2] += (double)rv.x * (double)rv.x;
                    v[3] += (double)rv.y * (double)rv.y;
                });
            tm.sync();
            team_sum<CW, 4>(tm, v, sh);
            for (int c = 0; c < 2; ++c)
                if (!done_c[c] && v[2 + c] <= tol_rel[c] * tol_rel[c] * rr0[c]) done_c[c] = true;
            const TI bx = (!done_c[0] && rz[0] > 0) ? (TI)(v[0] / rz[0]) : (TI)0;
            const TI by = (!done_c[1] && rz[1] > 0) ? (TI)(v[1] / rz[1]) : (TI)0;
            rz[0] = v[0];
            rz[1] = v[1];
            for_rows<kIlp>(tm, 
                ni, nj, -1,
                [&](int ii, int jj) {
                    const Pair<TI> z = L0.x[jj * ni + ii], pc = p[gid(ii, jj)];
                    return Pair<TI>{z.x + bx * pc.x, z.y + by * pc.y};
                },
                [&](int ii, int jj, const Pair<TI>& w) { p[gid(ii, jj)] = w; });
            tm.sync();
        }
        // x += e
        for_rows<kIlp>(tm, 
            ni, nj, -1,
            [&](int ii, int jj) {
                const long id = gid(ii, jj);
                const Pair<TI> ev = e[id];
                return Pair<double>{P.xnew[id] + (double)ev.x, P.ynew[id] + (double)ev.y};
            },
            [&](int ii, int jj, const Pair<double>& w) {
                const long id = gid(ii, jj);
                P.xnew[id] = w.x;
                P.ynew[id] = w.y;
            });
        tm.sync();
    }
    if (tm.tid() == 0) {
        P.stat_iters[sub] = iters;
        P.stat_outer[sub] = outer;
        P.stat_ok[sub] = ok;
        P.stat_res[sub] = rel;
    }
}

#ifndef SDD_SOLVE_SUB_ATTR
#define SDD_SOLVE_SUB_ATTR __forceinline__
#endif
template <typename TI, int CW>
__device__ SDD_SOLVE_SUB_ATTR void solve_sub(const Team<CW> tm, const SolveParams& P, int sub, double* sh);

template <typename TI>
__global__ void __launch_bounds__(kSolveThreads, kSolveMinBlocks) solve_kernel(const __grid_constant__ SolveParams P)
{
    __shared__ double sh[32 * 8 + 8];
    solve_sub<TI, 1>(Team<1>{0}, P, blockIdx.x, sh);
}

__global__ void __launch_bounds__(kSolveThreads) fe_kernel(const __grid_constant__ SolveParams P)
{
    __shared__ double sh[40];
    fe_body(P, blockIdx.x, sh);
}

// Batched problem record of CTA b: order[b] = (problem, subdomain) when given (largest
// subdomains first, so the longest CTAs start in the first wave), else problem p with
// sub_off[p] <= b < sub_off[p + 1].
__device__ __forceinline__ void batch_lookup(const SolveParams* probs, const int32_t* sub_off, const int2* order,
                                             int n, SolveParams& sp, int& sub)
{
    if (order) {
        const int2 o = order[blockIdx.x];
        sp = probs[o.x];
        sub = o.y;
        return;
    }
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sub_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    sp = probs[lo];
    sub = (int)blockIdx.x - sub_off[lo];
}

// Batched forward-Euler subdomains (CTAs of backward-Euler problems return at once).
__global__ void __launch_bounds__(kSolveThreads) fe_batch_kernel(const SolveParams* probs, const int32_t* sub_off,
                                                                 const int2* order, int n)
{
    __shared__ double sh[40];
    __shared__ SolveParams sp;
    __shared__ int sub;
    if (threadIdx.x == 0) batch_lookup(probs, sub_off, order, n, sp, sub);
    __syncthreads();
    if (sp.scheme == 1) fe_body(sp, sub, sh);
}

// Batched: CTA b solves the subdomain batch_lookup assigns it (launches without large subdomains;
// with them, solve_batch_items_kernel below).
template <typename TI>
__global__ void __launch_bounds__(kSolveThreads, kSolveMinBlocks) solve_batch_kernel(const SolveParams* probs,
                                                                       const int32_t* sub_off, const int2* order,
                                                                       int n)
{
    __shared__ double sh[32 * 8 + 8];
    __shared__ SolveParams sp;
    __shared__ int sub;
    if (threadIdx.x == 0) batch_lookup(probs, sub_off, order, n, sp, sub);
    __syncthreads();
    if (sp.scheme == 0) solve_sub<TI, 1>(Team<1>{0}, sp, sub, sh);  // forward-Euler problems: fe_batch_kernel
}

// The solve of one subdomain, called by every solve kernel.  Inlined into each kernel (measured
// 5 % faster on the 64-problem mix than one shared out-of-line copy, which spills at the call
// boundary); the same source and reduction order in every kernel give a subdomain the same bits in
// a single-problem launch, a batch and a served request (checked bitwise by the batch and serving
// tests).
template <typename TI, int CW>
__device__ SDD_SOLVE_SUB_ATTR void solve_sub(const Team<CW> tm, const SolveParams& P, int sub, double* sh)
{
    solve_body<TI, CW>(tm, P, sub, sh);
}

// Subdomains with at least kCoopUnknowns interior unknowns are solved by the kCoopWidth CTAs of
// a thread-block cluster (2048 threads on at least two SMs): rows, loops and reductions are spread
// over the cluster and every pass ends in a cluster barrier.  The
// team width is a function of the subdomain's size alone, so a subdomain gives the same bits in a
// single-problem launch, a batch and a served request.
template <typename TI>
__device__ __forceinline__ void solve_item(const SolveParams& sp, const SolveItem& it, double* sh)
{
    if (it.width == kCoopWidth) {
        const unsigned rank = cooperative_groups::this_cluster().block_rank();
        solve_sub<TI, kCoopWidth>(Team<kCoopWidth>{(int)rank}, sp, it.sub, sh);
    } else if (it.width == 1) {
        solve_sub<TI, 1>(Team<1>{0}, sp, it.sub, sh);
    }
}

// One work item per CTA (launch: items.size() CTAs in clusters of kCoopWidth).  A cooperative
// item fills a whole cluster (its kCoopWidth entries are the same); otherwise each CTA of the
// cluster solves its own subdomain, or none (width 0).
template <typename TI>
__global__ void __cluster_dims__(kCoopWidth, 1, 1) __launch_bounds__(kSolveThreads, kSolveMinBlocks)
    solve_items_kernel(const __grid_constant__ SolveParams P, const SolveItem* items)
{
    __shared__ double sh[32 * 8 + 8];
    solve_item<TI>(P, items[blockIdx.x], sh);
}

template <typename TI>
__global__ void __cluster_dims__(kCoopWidth, 1, 1) __launch_bounds__(kSolveThreads, kSolveMinBlocks)
    solve_batch_items_kernel(const SolveParams* probs, const SolveItem* items)
{
    __shared__ double sh[32 * 8 + 8];
    __shared__ SolveParams sp;
    const SolveItem it = items[blockIdx.x];
    if (threadIdx.x == 0 && it.width > 0) sp = probs[it.prob];
    __syncthreads();
    if (it.width > 0 && sp.scheme == 0) solve_item<TI>(sp, it, sh);
}

}  // namespace

std::vector<SolveItem> solve_items(const std::vector<std::pair<int64_t, int2>>& subs)
{
    std::vector<SolveItem> items;
    bool any = false;
    for (const auto& v : subs) any = any || v.first >= kCoopUnknowns;
    if (!any) return items;
    std::vector<SolveItem> pend;  // subdomains of one CTA each, waiting to fill a cluster
    for (const auto& v : subs) {
        if (v.first >= kCoopUnknowns) {
            for (int r = 0; r < kCoopWidth; ++r) items.push_back(SolveItem{v.second.x, v.second.y, kCoopWidth, 0});
        } else {
            pend.push_back(SolveItem{v.second.x, v.second.y, 1, 0});
            if ((int)pend.size() == kCoopWidth) {
                items.insert(items.end(), pend.begin(), pend.end());
                pend.clear();
            }
        }
    }
    if (!pend.empty()) {
        while ((int)pend.size() < kCoopWidth) pend.push_back(SolveItem{0, 0, 0, 0});
        items.insert(items.end(), pend.begin(), pend.end());
    }
    return items;
}

cudaError_t launch_solve_items(const SolveParams& P, const SolveItem* items, int n_items, bool fp64_inner,
                               cudaStream_t s)
{
    const long n = (long)P.nx * P.ny;
    faces_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(P, fp64_inner ? 1 : 0);
    if (n_items <= 0) return cudaGetLastError();
    if (fp64_inner)
        solve_items_kernel<double><<<n_items, kSolveThreads, 0, s>>>(P, items);
    else
        solve_items_kernel<float><<<n_items, kSolveThreads, 0, s>>>(P, items);
    return cudaGetLastError();
}

cudaError_t launch_solve_batch_items(const SolveParams* probs, const SolveItem* items, int n_items,
                                     bool fp64_inner, cudaStream_t s)
{
    if (n_items <= 0) return cudaSuccess;
    if (fp64_inner)
        solve_batch_items_kernel<double><<<n_items, kSolveThreads, 0, s>>>(probs, items);
    else
        solve_batch_items_kernel<float><<<n_items, kSolveThreads, 0, s>>>(probs, items);
    return cudaGetLastError();
}

cudaError_t launch_faces_batch(const SolveParams* probs, const int32_t* blk_off, int n, int total_blocks,
                               bool fp64_inner, cudaStream_t s)
{
    faces_batch_kernel<<<total_blocks, 256, 0, s>>>(probs, blk_off, n, fp64_inner ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_faces(const SolveParams& P, bool fp64_inner, cudaStream_t s)
{
    const long n = (long)P.nx * P.ny;
    faces_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(P, fp64_inner ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_solve_batch(const SolveParams* probs, const int32_t* sub_off, int n, int total_subs,
                               bool fp64_inner, cudaStream_t s, bool any_be, bool any_fe, const int2* order)
{
    if (total_subs <= 0) return cudaSuccess;
    if (any_be) {
        if (fp64_inner)
            solve_batch_kernel<double><<<total_subs, kSolveThreads, 0, s>>>(probs, sub_off, order, n);
        else
            solve_batch_kernel<float><<<total_subs, kSolveThreads, 0, s>>>(probs, sub_off, order, n);
    }
    if (any_fe) fe_batch_kernel<<<total_subs, kSolveThreads, 0, s>>>(probs, sub_off, order, n);
    return cudaGetLastError();
}

cudaError_t launch_solve(const SolveParams& P, bool fp64_inner, cudaStream_t s)
{
    const long n = (long)P.nx * P.ny;
    faces_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(P, fp64_inner ? 1 : 0);
    const int nsub = P.px * P.py;
    if (P.scheme == 1)
        fe_kernel<<<nsub, kSolveThreads, 0, s>>>(P);
    else if (fp64_inner)
        solve_kernel<double><<<nsub, kSolveThreads, 0, s>>>(P);
    else
        solve_kernel<float><<<nsub, kSolveThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace sdd
