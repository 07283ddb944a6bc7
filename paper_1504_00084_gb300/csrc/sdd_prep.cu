// Monitor preparation and Dirichlet-data scatter (grid-sized, HBM/L2-bound, negligible next
// to the path kernel).
//
//   prep_omega_kernel : omega at every node on the current mesh at t^n (Sec. 2, Sec. 3.2),
//                       FP64; periodic wrap nodes evaluate their canonical node so they
//                       repeat it bit for bit.
//   prep_pack_kernel  : finite-difference gradient of omega in the computational
//                       coordinates (Sec. 3.4), the packed {omega, omega_xi, omega_eta}
//                       records in the path precision (FP64: one per node; FP32: the four
//                       corners of every node's cell), and the previous mesh
//                       as a displacement from the identity.
//   scatter kernels   : the new mesh's Dirichlet data -- physical boundary (identity) and
//                       interface estimates with periodic offsets (Sec. 3.5).
//   face kernel       : face coefficients of the backward-Euler subdomain systems.
//
// The prep arithmetic uses explicit round-to-nearest intrinsics (no fused multiply-add), so
// the FP64 monitor record is reproducible independently of compiler contraction choices.
#include <math.h>

#include "sdd_internal.cuh"

namespace sdd {

namespace {

constexpr int kMonGauss = 1, kMonFront = 2, kMonRings = 4;  // otherwise bumps (3) or nodal (0)

__device__ __forceinline__ double min_image(double d, double L, int periodic)
{
    return periodic ? d - L * floor(d / L + 0.5) : d;
}

__device__ double monitor_value(const PrepParams& P, double x, double y, double t)
{
    const double* q = P.params;
    if (P.kind == kMonGauss) {
        const double dx = min_image(x - q[2], P.Lx, P.periodic);
        const double dy = min_image(y - q[3], P.Ly, P.periodic);
        return sqrt(1.0 + q[0] * exp(-q[1] * (dx * dx + dy * dy)));
    }
    if (P.kind == kMonFront) {
        const double dx = min_image(x - q[4], P.Lx, P.periodic);
        const double dy = min_image(y - q[5], P.Ly, P.periodic);
        const double r = sqrt(dx * dx + dy * dy);
        const double u = tanh(q[1] * (r - q[2] - q[3] * t));
        const double g = q[1] * (1.0 - u * u);      // |grad u|
        return sqrt(1.0 + q[0] * g * g);
    }
    if (P.kind == kMonRings) {                       // sum of tanh rings (five-ring problem)
        double gx = 0.0, gy = 0.0;
        for (int b = 3; b + 1 < P.n_params; b += 2) {
            const double dx = min_image(x - q[b], P.Lx, P.periodic);
            const double dy = min_image(y - q[b + 1], P.Ly, P.periodic);
            const double uk = tanh(q[1] * (dx * dx + dy * dy - q[2]));
            const double f = q[1] * (1.0 - uk * uk) * 2.0;
            gx += f * dx;
            gy += f * dy;
        }
        return sqrt(1.0 + q[0] * (gx * gx + gy * gy));
    }
    double w = 1.0;                                  // bumps
    for (int b = 0; b + 3 < P.n_params; b += 4) {
        const double dx = min_image(x - q[b + 2], P.Lx, P.periodic);
        const double dy = min_image(y - q[b + 3], P.Ly, P.periodic);
        w += q[b] * exp(-(dx * dx + dy * dy) / (q[b + 1] * q[b + 1]));
    }
    return w;
}

// Monitor on the current mesh at every node (the body of one block of blocks nb).
__device__ __forceinline__ void prep_omega_body(const PrepParams& P, int blk, int nb)
{
    const int n = P.nx * P.ny;
    const double t = P.t_dev ? *P.t_dev : P.t;
    for (int id = blk * blockDim.x + threadIdx.x; id < n; id += nb * blockDim.x) {
        const int i = id % P.nx, j = id / P.nx;
        const int ci = P.periodic ? i % (P.nx - 1) : i;
        const int cj = P.periodic ? j % (P.ny - 1) : j;
        const int c = cj * P.nx + ci;
        P.om64[id] = P.kind == 0 ? P.omega_in[c] : monitor_value(P, P.x[c], P.y[c], t);
    }
}

__global__ void prep_omega_kernel(const PrepParams P) { prep_omega_body(P, blockIdx.x, gridDim.x); }

// d f / d s along one grid line at index i of n nodes: central differences in the interior,
// one-sided second order at Dirichlet ends, wrapped when periodic; factor c = (n - 1) / 2.
__device__ __forceinline__ double fd_line(const double* f, long stride, int i, int n, int periodic)
{
    const double c = 0.5 * (double)(n - 1);
    if (periodic) {
        const int m = n - 1;
        const int ii = i % m;
        const int ip = (ii + 1) % m, im = (ii + m - 1) % m;
        return __dmul_rn(__dsub_rn(f[ip * stride], f[im * stride]), c);
    }
    if (i == 0)
        return __dmul_rn(__dsub_rn(__dadd_rn(__dmul_rn(-3.0, f[0]), __dmul_rn(4.0, f[stride])),
                                   f[2 * stride]), c);
    if (i == n - 1)
        return __dmul_rn(__dsub_rn(__dadd_rn(__dmul_rn(3.0, f[(long)(n - 1) * stride]),
                                             __dmul_rn(-4.0, f[(long)(n - 2) * stride])),
                                   -f[(long)(n - 3) * stride]), c);
    return __dmul_rn(__dsub_rn(f[(long)(i + 1) * stride], f[(long)(i - 1) * stride]), c);
}

template <typename T>
__device__ __forceinline__ void prep_pack_body(const PrepParams& P, int blk, int nb)
{
    const int n = P.nx * P.ny;
    Mon4<T>* mon = static_cast<Mon4<T>*>(P.mon);
    Disp2<T>* disp = static_cast<Disp2<T>*>(P.disp);
    for (int id = blk * blockDim.x + threadIdx.x; id < n; id += nb * blockDim.x) {
        const int i = id % P.nx, j = id / P.nx;
        const double w = P.om64[id];
        const double wx = fd_line(P.om64 + (long)j * P.nx, 1, i, P.nx, P.periodic);
        const double we = fd_line(P.om64 + i, P.nx, j, P.ny, P.periodic);
        P.wxi64[id] = wx;
        P.weta64[id] = we;
        const Mon4<T> rec{(T)w, (T)wx, (T)we, (T)0};
        if constexpr (sizeof(T) == 8) {
            mon[id] = rec;
        } else {  // FP32 cell records (corners clamped to the grid): every slot whose corner is this node
            const int nx = P.nx, ny = P.ny;
            const bool lx = i == nx - 1, ly = j == ny - 1;
            Mon4<T>* c0 = mon + 4 * (long)id;  // cell (i, j)
            c0[0] = rec;
            if (lx) c0[1] = rec;
            if (ly) c0[2] = rec;
            if (lx && ly) c0[3] = rec;
            if (i > 0) {
                Mon4<T>* cl = c0 - 4;  // cell (i - 1, j)
                cl[1] = rec;
                if (ly) cl[3] = rec;
            }
            if (j > 0) {
                Mon4<T>* cd = c0 - 4 * (long)nx;  // cell (i, j - 1)
                cd[2] = rec;
                if (lx) cd[3] = rec;
                if (i > 0) cd[-4 + 3] = rec;  // cell (i - 1, j - 1)
            }
        }
        const int ci = P.periodic ? i % (P.nx - 1) : i;
        const int cj = P.periodic ? j % (P.ny - 1) : j;
        const int c = cj * P.nx + ci;
        const double xi = (double)ci / (double)(P.nx - 1);
        const double eta = (double)cj / (double)(P.ny - 1);
        const double X = __dsub_rn(P.x[c], __dmul_rn(P.Lx, xi));
        const double Y = __dsub_rn(P.y[c], __dmul_rn(P.Ly, eta));
        disp[id] = Disp2<T>{(T)X, (T)Y};
        // the monitor must be positive and everything finite (Sec. 2: omega > 0)
        if (P.bad && !(w > 0.0 && isfinite(w) && isfinite(wx) && isfinite(we) && isfinite(X) && isfinite(Y)))
            atomicOr(P.bad, 1);
    }
}

template <typename T>
__global__ void prep_pack_kernel(const PrepParams P) { prep_pack_body<T>(P, blockIdx.x, gridDim.x); }

__global__ void shift_kernel(const int2* nodes, int M, int nx, const double* x, const double* y,
                             double* shift)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int2 ij = nodes[m];
    shift[2 * m] = x[(long)ij.y * nx + ij.x];
    shift[2 * m + 1] = y[(long)ij.y * nx + ij.x];
}

__device__ __forceinline__ void scatter_boundary_body(int nx, int ny, double Lx, double Ly, double* xnew,
                                                      double* ynew, const double* bnd, int blk, int nb)
{
    const int n = nx * ny;
    for (int id = blk * blockDim.x + threadIdx.x; id < n; id += nb * blockDim.x) {
        const int i = id % nx, j = id / nx;
        if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) {
            double vx = Lx * ((double)i / (double)(nx - 1));
            double vy = Ly * ((double)j / (double)(ny - 1));
            if (bnd) {  // moving boundary: tangential components from the 1-D step
                if (j == 0) vx = bnd[i];
                else if (j == ny - 1) vx = bnd[nx + i];
                if (i == 0) vy = bnd[2 * nx + j];
                else if (i == nx - 1) vy = bnd[2 * nx + ny + j];
            }
            xnew[id] = vx;
            ynew[id] = vy;
        }
    }
}

__global__ void scatter_boundary_kernel(int nx, int ny, double Lx, double Ly, double* xnew,
                                        double* ynew, const double* bnd)
{
    scatter_boundary_body(nx, ny, Lx, Ly, xnew, ynew, bnd, blockIdx.x, gridDim.x);
}

// One backward-Euler step of the 1-D generator along each side of a Dirichlet domain (Sec. 2):
// side s (thread s) carries the tangential coordinate b_k at its n nodes -- x along eta = 0
// (s = 0) and eta = 1 (s = 1), y along xi = 0 (s = 2) and xi = 1 (s = 3) -- and solves
//   d_k b_k + r sum_{nb = k +- 1} c_{k,nb} (b_k - b_nb) = d_k b^n_k,  k = 1 .. n-2,
//   c_{k,k+1} = (omega_k + omega_{k+1}) / 2 / h^2,  d_k = 1 (form 0) or omega_k (form 1),
// with the corner values fixed, by the tridiagonal (Thomas) sweeps; the system is a
// diagonally dominant M-matrix.
template <typename T>
__device__ __forceinline__ void boundary_body(const PrepParams& P)
{
    const int s = threadIdx.x;
    if (s >= 4) return;
    const int nx = P.nx, ny = P.ny;
    const int n = s < 2 ? nx : ny;
    const long off = s == 0 ? 0 : s == 1 ? nx : s == 2 ? 2L * nx : 2L * nx + ny;
    auto id = [&](int k) -> long {
        return s == 0 ? k : s == 1 ? (long)(ny - 1) * nx + k : s == 2 ? (long)k * nx : (long)k * nx + nx - 1;
    };
    auto coord = [&](int k) -> double { return s < 2 ? P.x[id(k)] : P.y[id(k)]; };
    double* b = P.bnd64 + off;
    double* cp = P.bnd_scratch + 2 * off;
    double* dp = cp + n;
    const double h2 = (double)(n - 1) * (double)(n - 1);
    b[0] = coord(0);
    b[n - 1] = coord(n - 1);
    for (int k = 1; k <= n - 2; ++k) {
        const double w = P.om64[id(k)];
        const double cw = __dmul_rn(P.r, __dmul_rn(__dmul_rn(0.5, __dadd_rn(w, P.om64[id(k - 1)])), h2));
        const double ce = __dmul_rn(P.r, __dmul_rn(__dmul_rn(0.5, __dadd_rn(w, P.om64[id(k + 1)])), h2));
        const double d = P.form == 1 ? w : 1.0;
        const double diag = __dadd_rn(__dadd_rn(d, cw), ce);
        double rhs = __dmul_rn(d, coord(k));
        double lower = -cw, upper = -ce;
        if (k == 1) { rhs = __dadd_rn(rhs, __dmul_rn(cw, b[0])); lower = 0.0; }
        if (k == n - 2) { rhs = __dadd_rn(rhs, __dmul_rn(ce, b[n - 1])); upper = 0.0; }
        const double m = k == 1 ? diag : __dsub_rn(diag, __dmul_rn(lower, cp[k - 1]));
        cp[k] = __ddiv_rn(upper, m);
        dp[k] = __ddiv_rn(k == 1 ? rhs : __dsub_rn(rhs, __dmul_rn(lower, dp[k - 1])), m);
    }
    if (n > 2) b[n - 2] = dp[n - 2];
    for (int k = n - 3; k >= 1; --k) b[k] = __dsub_rn(dp[k], __dmul_rn(cp[k], b[k + 1]));
    T* bt = static_cast<T*>(P.bnd) + off;
    for (int k = 0; k < n; ++k) bt[k] = (T)b[k];
}

template <typename T>
__global__ void boundary_kernel(const PrepParams P) { boundary_body<T>(P); }

__device__ __forceinline__ void scatter_iface_one(int nx, int ny, int periodic, double Lx, double Ly,
                                                  const int2* nodes, int m, const double* est, double* xnew,
                                                  double* ynew)
{
    const int2 ij = nodes[m];
    const double vx = est[2 * m], vy = est[2 * m + 1];
    const long id = (long)ij.y * nx + ij.x;
    xnew[id] = vx;
    ynew[id] = vy;
    if (periodic) {
        if (ij.x == 0) {
            xnew[id + nx - 1] = vx + Lx;
            ynew[id + nx - 1] = vy;
        }
        if (ij.y == 0) {
            const long w = (long)(ny - 1) * nx + ij.x;
            xnew[w] = vx;
            ynew[w] = vy + Ly;
        }
        if (ij.x == 0 && ij.y == 0) {
            const long w = (long)(ny - 1) * nx + nx - 1;
            xnew[w] = vx + Lx;
            ynew[w] = vy + Ly;
        }
    }
}

__global__ void scatter_iface_kernel(int nx, int ny, int periodic, double Lx, double Ly,
                                     const int2* nodes, int M, const double* est, double* xnew,
                                     double* ynew)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    scatter_iface_one(nx, ny, periodic, Lx, Ly, nodes, m, est, xnew, ynew);
}

// ---------------------------------------------------------------------------------------
// Batched forms: one launch over the problems of a batch.  Grid-sized work gives problem i the
// blocks blk_off[i] .. blk_off[i + 1] - 1 (each problem its own block count, as its single-problem
// launch would have); node work runs over the batch's concatenated nodes.  Every node computes
// what the single-problem kernels compute for it.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int batch_problem_of_block(const int32_t* blk_off, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void prep_omega_batch_kernel(const BatchRec* R, const int32_t* blk_off, int n)
{
    const int i = batch_problem_of_block(blk_off, n, blockIdx.x);
    const int blk = blockIdx.x - blk_off[i], nb = blk_off[i + 1] - blk_off[i];
    if (blk == 0 && threadIdx.x == 0 && R[i].prep.bad) *R[i].prep.bad = 0;  // before the pack launch
    prep_omega_body(R[i].prep, blk, nb);
}

template <typename T>
__global__ void prep_pack_batch_kernel(const BatchRec* R, const int32_t* blk_off, int n)
{
    const int i = batch_problem_of_block(blk_off, n, blockIdx.x);
    prep_pack_body<T>(R[i].prep, blockIdx.x - blk_off[i], blk_off[i + 1] - blk_off[i]);
}

template <typename T>
__global__ void boundary_batch_kernel(const BatchRec* R)
{
    const PrepParams& P = R[blockIdx.x].prep;
    if (P.moving_boundary && !P.periodic) boundary_body<T>(P);
}

__global__ void shift_batch_kernel(const BatchRec* R, const int32_t* node_prob, int M, double* shift)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M) return;
    const BatchRec& r = R[node_prob[g]];
    const int2 ij = r.nodes[g - r.node_offset];
    shift[2 * g] = r.prep.x[(long)ij.y * r.prep.nx + ij.x];
    shift[2 * g + 1] = r.prep.y[(long)ij.y * r.prep.nx + ij.x];
}

__global__ void scatter_boundary_batch_kernel(const BatchRec* R, const int32_t* blk_off, int n)
{
    const int i = batch_problem_of_block(blk_off, n, blockIdx.x);
    const BatchRec& r = R[i];
    if (r.prep.periodic) return;
    scatter_boundary_body(r.prep.nx, r.prep.ny, r.prep.Lx, r.prep.Ly, r.xnew, r.ynew,
                          r.prep.moving_boundary ? r.prep.bnd64 : nullptr, blockIdx.x - blk_off[i],
                          blk_off[i + 1] - blk_off[i]);
}

__global__ void scatter_iface_batch_kernel(const BatchRec* R, const int32_t* node_prob, int M, const double* est)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M) return;
    const BatchRec& r = R[node_prob[g]];
    scatter_iface_one(r.prep.nx, r.prep.ny, r.prep.periodic, r.prep.Lx, r.prep.Ly, r.nodes, g - r.node_offset,
                      est + 2 * (size_t)r.node_offset, r.xnew, r.ynew);
}

// x <- x^{n+1}, y <- y^{n+1} of every problem (the step's last launch)
__global__ void copy_back_batch_kernel(const BatchRec* R, const int32_t* blk_off, int n)
{
    const int i = batch_problem_of_block(blk_off, n, blockIdx.x);
    const BatchRec& r = R[i];
    const int nb = blk_off[i + 1] - blk_off[i];
    const long N = (long)r.prep.nx * r.prep.ny;
    double* x = const_cast<double*>(r.prep.x);
    double* y = const_cast<double*>(r.prep.y);
    for (long id = (long)(blockIdx.x - blk_off[i]) * blockDim.x + threadIdx.x; id < N; id += (long)nb * blockDim.x) {
        x[id] = r.xnew[id];
        y[id] = r.ynew[id];
    }
}

// Geometric quality Q = tr(J^T J) / (2 |det J|) of every cell (Eq. 8), J from the mean of the
// cell's two xi-edges and two eta-edges; then the maximum and mean over the cells.
__global__ void quality_kernel(int nx, int ny, const double* x, const double* y, double* q)
{
    const long nc = (long)(nx - 1) * (ny - 1);
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < nc; c += (long)gridDim.x * blockDim.x) {
        const int i = (int)(c % (nx - 1)), j = (int)(c / (nx - 1));
        const long a = (long)j * nx + i, b = a + 1, d = a + nx, e = d + 1;
        const double x_xi = 0.5 * ((x[b] - x[a]) + (x[e] - x[d]));
        const double y_xi = 0.5 * ((y[b] - y[a]) + (y[e] - y[d]));
        const double x_eta = 0.5 * ((x[d] - x[a]) + (x[e] - x[b]));
        const double y_eta = 0.5 * ((y[d] - y[a]) + (y[e] - y[b]));
        const double tr = x_xi * x_xi + y_xi * y_xi + x_eta * x_eta + y_eta * y_eta;
        q[c] = 0.5 * tr / fabs(x_xi * y_eta - x_eta * y_xi);
    }
}

__global__ void max_mean_kernel(long n, const double* v, double* out)
{
    __shared__ double smax[32], ssum[32];
    double m = -INFINITY, s = 0.0;
    for (long k = threadIdx.x; k < n; k += blockDim.x) {
        m = fmax(m, v[k]);
        s += v[k];
    }
    for (int off = 16; off > 0; off >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        s += __shfl_xor_sync(0xffffffffu, s, off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { smax[w] = m; ssum[w] = s; }
    __syncthreads();
    if (threadIdx.x == 0) {  // holds warp 0's totals; add the other warps in order
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { m = fmax(m, smax[k]); s += ssum[k]; }
        out[0] = m;
        out[1] = s / (double)n;
    }
}

inline int blocks_for(long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_prep(const PrepParams& P, cudaStream_t s)
{
    const long n = (long)P.nx * P.ny;
    const int threads = 256;
    const int blocks = blocks_for(n, threads);
    prep_omega_kernel<<<blocks, threads, 0, s>>>(P);
    if (P.precision == 0)
        prep_pack_kernel<double><<<blocks, threads, 0, s>>>(P);
    else
        prep_pack_kernel<float><<<blocks, threads, 0, s>>>(P);
    if (P.moving_boundary && !P.periodic) {
        if (P.precision == 0)
            boundary_kernel<double><<<1, 32, 0, s>>>(P);
        else
            boundary_kernel<float><<<1, 32, 0, s>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_quality(int nx, int ny, const double* x, const double* y, double* q, double* stats,
                           cudaStream_t s)
{
    const long nc = (long)(nx - 1) * (ny - 1);
    quality_kernel<<<blocks_for(nc, 256), 256, 0, s>>>(nx, ny, x, y, q);
    max_mean_kernel<<<1, 1024, 0, s>>>(nc, q, stats);
    return cudaGetLastError();
}

cudaError_t launch_shift(const int2* nodes, int M, int nx, const double* x, const double* y,
                         double* shift, cudaStream_t s)
{
    shift_kernel<<<blocks_for(M, 256), 256, 0, s>>>(nodes, M, nx, x, y, shift);
    return cudaGetLastError();
}

cudaError_t launch_scatter(int nx, int ny, int periodic, double Lx, double Ly, const int2* nodes,
                           int M, const double* est, double* xnew, double* ynew, cudaStream_t s,
                           const double* bnd64)
{
    if (!periodic)
        scatter_boundary_kernel<<<blocks_for((long)nx * ny, 256), 256, 0, s>>>(nx, ny, Lx, Ly, xnew,
                                                                               ynew, bnd64);
    if (M > 0)
        scatter_iface_kernel<<<blocks_for(M, 256), 256, 0, s>>>(nx, ny, periodic, Lx, Ly, nodes, M, est,
                                                                xnew, ynew);
    return cudaGetLastError();
}

}  // namespace sdd

namespace sdd {

int batch_blocks(long n_nodes) { return blocks_for(n_nodes, 256); }

cudaError_t launch_prep_batch(const BatchRec* R, const int32_t* blk_off, int n, int total_blocks, bool fp64,
                              bool any_moving, cudaStream_t s)
{
    prep_omega_batch_kernel<<<total_blocks, 256, 0, s>>>(R, blk_off, n);
    if (fp64)
        prep_pack_batch_kernel<double><<<total_blocks, 256, 0, s>>>(R, blk_off, n);
    else
        prep_pack_batch_kernel<float><<<total_blocks, 256, 0, s>>>(R, blk_off, n);
    if (any_moving) {
        if (fp64)
            boundary_batch_kernel<double><<<n, 32, 0, s>>>(R);
        else
            boundary_batch_kernel<float><<<n, 32, 0, s>>>(R);
    }
    return cudaGetLastError();
}

cudaError_t launch_shift_batch(const BatchRec* R, const int32_t* node_prob, int M, double* shift, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    shift_batch_kernel<<<blocks_for(M, 256), 256, 0, s>>>(R, node_prob, M, shift);
    return cudaGetLastError();
}

cudaError_t launch_scatter_batch(const BatchRec* R, const int32_t* blk_off, int n, int total_blocks,
                                 const int32_t* node_prob, int M, const double* est, cudaStream_t s)
{
    scatter_boundary_batch_kernel<<<total_blocks, 256, 0, s>>>(R, blk_off, n);
    if (M > 0) scatter_iface_batch_kernel<<<blocks_for(M, 256), 256, 0, s>>>(R, node_prob, M, est);
    return cudaGetLastError();
}

cudaError_t launch_copy_back_batch(const BatchRec* R, const int32_t* blk_off, int n, int total_blocks, cudaStream_t s)
{
    copy_back_batch_kernel<<<total_blocks, 256, 0, s>>>(R, blk_off, n);
    return cudaGetLastError();
}

}  // namespace sdd
