// Interface Monte Carlo of the SDD mesh generator (Sec. 3.4), sm_103a.
//
// Work decomposition.  A round gives every active interface node a chunk of consecutive
// path indices; chunks are cut into tasks of kPathsPerTask paths.  A persistent grid of warps
// pulls tasks from an atomic counter.  Inside a task each lane runs one path at a time and,
// when its path ends (exit or K substeps), immediately takes the next unused path index of
// the task (ballot + popc), so the 32 lanes stay busy through paths of very different
// lengths.  A path that completes its K substeps parks its final point in a per-warp
// shared-memory queue; the warp evaluates the bicubic terminal values 32 at a time, one per
// lane, instead of stalling on that long branch whenever any single lane finishes.  Exits are
// queued the same way (proposed point and bridge side), and their exit points, boundary values
// and sums are formed 32 at a time rather than on the few lanes whose path just ended.  The
// assignment of path indices to lanes depends only on the paths' own lengths,
// so a task's partial sums are a deterministic function of (node, path range) and are
// independent of scheduling and of which other problems or nodes share the launch.
//
// Per substep and lane: one Philox4x32-10 call keyed by the seed with counter
// (k, p, m, n) -> Box-Muller normals (words 0, 1; FP32 angle through sincos_2pi) and the
// bridge uniform (word 2); bilinear
// gather of {omega, omega_xi, omega_eta} from the packed monitor (read-only cache; the
// record of a node is one 16-byte (FP32) or 32-byte (FP64) load); Euler-Maruyama update
// (Eq. 7); endpoint and Brownian-bridge exit tests.  Terminal values: the boundary mesh at
// the exit point, or the Keys-bicubic previous mesh at the final point (Eq. 5a, Eq. 6).
//
// Reductions: per-lane sums of the shifted values (FP64, or Kahan-compensated FP32), a
// fixed xor-shuffle tree per task, one slot per task, then one warp per node adds its slots
// in task order.  No floating-point atomics: results are bitwise reproducible.
#include <math.h>

#include "sdd_internal.cuh"

namespace sdd {

namespace {

constexpr int kMcThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
#ifndef SDD_MC_MIN_BLOCKS
#define SDD_MC_MIN_BLOCKS 4   // FP32: resident blocks per SM asked of the register allocator (64 registers)
#endif
// FP64 paths need more registers; two resident blocks keep them out of local memory.  Other block
// sizes (batched launches, chosen by sdd_batch_tune) keep the same threads per SM.
template <typename T, int TPB = kMcThreads>
constexpr int mc_min_blocks() { return (sizeof(T) == 8 ? 2 : SDD_MC_MIN_BLOCKS) * kMcThreads / TPB; }

__device__ __forceinline__ float dlog(float x) { return logf(x); }
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dfloor(float x) { return floorf(x); }
__device__ __forceinline__ double dfloor(double x) { return floor(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }
__device__ __forceinline__ float dmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double dmin(double a, double b) { return fmin(a, b); }

}  // namespace

// Gather-index check, compiled in only with SDD_BOUNDS_CHECK: an index outside [0, n) is counted
// in g_bounds_violations and replaced by 0, so the load stays inside its array.  The normal
// build returns the index unchanged.
#ifdef SDD_BOUNDS_CHECK
__device__ unsigned long long g_bounds_violations;
template <typename I>
__device__ __forceinline__ I checked(I i, long n)
{
    if ((long)i < 0 || (long)i >= n) {
        atomicAdd(&g_bounds_violations, 1ull);
        return (I)0;
    }
    return i;
}
// the same for a pointer into the n-element array at base
template <typename V>
__device__ __forceinline__ const V* checked_ptr(const V* q, const V* base, long n)
{
    const long i = q - base;
    if (i < 0 || i >= n) {
        atomicAdd(&g_bounds_violations, 1ull);
        return base;
    }
    return q;
}
#else
template <typename I>
__device__ __forceinline__ I checked(I i, long) { return i; }
template <typename V>
__device__ __forceinline__ const V* checked_ptr(const V* q, const V*, long) { return q; }
#endif

namespace {

// sin(2 pi u), cos(2 pi u) for u in (0, 1).  t = 4u is exact; with q = rint(t) and r = t - q
// (exact, |r| <= 1/2) the angle is (pi/2)(q + r), so q mod 4 permutes and signs the sine and
// cosine of (pi/2) r, taken from their Taylor series: coefficients (pi/2)^n / n! rounded to
// FP32, truncated after r^9 (sine) and r^10 (cosine), where the remainders are below 2e-9 at
// |r| = 1/2.  Measured error of the FP32 evaluation: below 0.75 ulp of 1 over the whole range.
__device__ __forceinline__ void sincos_2pi(float u, float* sn, float* cs)
{
    const float t = 4.0f * u;
    // q = rint(t) from the rounding of t + 1.5 2^23 (unit spacing there, ties to even, as rintf);
    // the sum's low mantissa bits hold q itself, so q mod 4 needs no conversion
    const float big = t + 0x1.8p23f;
    const float q = big - 0x1.8p23f;
    const int qint = __float_as_int(big);
    const float r = t - q;
    const float r2 = r * r;
    float ps = 0x1.507834p-13f;                 // (pi/2)^9 / 9!
    ps = fmaf(ps, r2, -0x1.32d2ccp-8f);         // -(pi/2)^7 / 7!
    ps = fmaf(ps, r2, 0x1.466bc6p-4f);          // (pi/2)^5 / 5!
    ps = fmaf(ps, r2, -0x1.4abbcep-1f);         // -(pi/2)^3 / 3!
    ps = fmaf(ps, r2, 0x1.921fb6p+0f);          // pi/2
    ps *= r;
    float pc = -0x1.a6d1f2p-16f;                // -(pi/2)^10 / 10!
    pc = fmaf(pc, r2, 0x1.e1f506p-11f);         // (pi/2)^8 / 8!
    pc = fmaf(pc, r2, -0x1.55d3c8p-6f);         // -(pi/2)^6 / 6!
    pc = fmaf(pc, r2, 0x1.03c1f0p-2f);          // (pi/2)^4 / 4!
    pc = fmaf(pc, r2, -0x1.3bd3ccp+0f);         // -(pi/2)^2 / 2!
    pc = fmaf(pc, r2, 1.0f);
    const int qi = qint & 3;
    float s_ = (qi & 1) ? pc : ps;
    float c_ = (qi & 1) ? ps : pc;
    if (qi & 2) s_ = -s_;           // quadrants 2, 3
    if ((qi + 1) & 2) c_ = -c_;     // quadrants 1, 2
    *sn = s_;
    *cs = c_;
}

template <typename T> struct Consts;
template <> struct Consts<double> {
    static constexpr double two_pi = 6.28318530717958647692;
    // exp(-a) below this argument's reach leaves 1 - exp(-a) == 1 exactly (and cannot be the
    // largest crossing probability of an exiting path), so the exponential is skipped.
    static constexpr double bridge_skip = 40.0;
};

__device__ __forceinline__ Mon4<float> load_mon(const Mon4<float>* p)
{
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return Mon4<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Mon4<double> load_mon(const Mon4<double>* p)
{
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return Mon4<double>{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ Disp2<float> load_disp(const Disp2<float>* p)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return Disp2<float>{v.x, v.y};
}
__device__ __forceinline__ Disp2<double> load_disp(const Disp2<double>* p)
{
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return Disp2<double>{v.x, v.y};
}

// Cell and in-cell offset of coordinate s on an n-node line over [0, 1]; periodic lines repeat
// with period 1 over n - 1 distinct nodes.
template <typename T>
__device__ __forceinline__ void locate(int n, int periodic, T s, int& cell, T& frac)
{
    const T u = s * (T)(n - 1);
    const T fl = dfloor(u);
    int c = (int)fl;
    if (periodic) {
        const int m = n - 1;
        c %= m;
        if (c < 0) c += m;
        frac = u - fl;
    } else {
        c = c < 0 ? 0 : (c > n - 2 ? n - 2 : c);
        frac = u - (T)c;
    }
    cell = c;
}

// Bilinear interpolation of the packed monitor at (xi, eta) (Sec. 3.4).
// FP32 cell and offset of coordinate s in [0, 1] on a Dirichlet n-node line, without
// conversions: v = min(s (n - 1), n - 3/2) has floor(v) = the clamped cell (cell n - 2 for
// s = 1), and v + 2^23 rounded down holds floor(v) in its low mantissa bits (unit spacing
// there), so it is the float 2^23 + cell, exactly; the returned bits are 0x4B000000 + cell.
// Paths inside the unit square only (a Dirichlet path leaves at its first step outside).
__device__ __forceinline__ uint32_t locate_dirichlet(int n, float s, float& frac)
{
    const float u = s * (float)(n - 1);
    const float v = fminf(u, (float)(n - 1) - 0.5f);
    const float t = __fadd_rd(v, 0x1.0p23f);
    frac = u - (t - 0x1.0p23f);
    return (uint32_t)__float_as_int(t);
}

template <typename T>
__device__ __forceinline__ void monitor_at(const McProblem<T>& P, T xi, T eta, T& w, T& wx, T& we)
{
    T fx, fy;
    int base;  // grids hold at most 2^28 nodes
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (!P.periodic) {
            const uint32_t bi = locate_dirichlet(P.nx, xi, fx);
            const uint32_t bj = locate_dirichlet(P.ny, eta, fy);
            base = (int)(bj * (uint32_t)P.nx + bi - P.cell_bias);
            done = true;
        }
    }
    if (!done) {
        int i, j;
        locate(P.nx, P.periodic, xi, i, fx);
        locate(P.ny, P.periodic, eta, j, fy);
        base = j * P.nx + i;
    }
    const long N = (long)P.nx * P.ny;
    const Mon4<T> a = load_mon(P.mon + checked(base, N)), b = load_mon(P.mon + checked(base + 1, N));
    const Mon4<T> c = load_mon(P.mon + checked(base + P.nx, N));
    const Mon4<T> d = load_mon(P.mon + checked(base + P.nx + 1, N));
    if constexpr (sizeof(T) == 4) {
        // paired FP32 arithmetic (one instruction for two lanes of work), operation for
        // operation the contraction of the plain expressions below: bit-identical results
        const float2 g = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-fx, -fy));
        const float2 wa = __fmul2_rn(make_float2(g.x, fx), make_float2(g.y, g.y));  // w00, w10
        const float2 wb = __fmul2_rn(make_float2(g.x, fx), make_float2(fy, fy));    // w01, w11
        float2 t = __fmul2_rn(make_float2(wa.y, wa.y), make_float2(b.w, b.wx));
        t = __ffma2_rn(make_float2(wa.x, wa.x), make_float2(a.w, a.wx), t);
        t = __ffma2_rn(make_float2(wb.x, wb.x), make_float2(c.w, c.wx), t);
        t = __ffma2_rn(make_float2(wb.y, wb.y), make_float2(d.w, d.wx), t);
        w = t.x;
        wx = t.y;
        we = fmaf(wb.y, d.we, fmaf(wb.x, c.we, fmaf(wa.x, a.we, wa.y * b.we)));
    } else {
        const T gx = 1 - fx, gy = 1 - fy;
        const T w00 = gx * gy, w10 = fx * gy, w01 = gx * fy, w11 = fx * fy;
        w = w00 * a.w + w10 * b.w + w01 * c.w + w11 * d.w;
        wx = w00 * a.wx + w10 * b.wx + w01 * c.wx + w11 * d.wx;
        we = w00 * a.we + w10 * b.we + w01 * c.we + w11 * d.we;
    }
}

// Keys (1981) cubic-convolution kernel, a = -1/2.
template <typename T>
__device__ __forceinline__ T keys_kernel(T s)
{
    const T a = (T)-0.5;
    s = dabs(s);
    if (s <= 1) return (a + 2) * s * s * s - (a + 3) * s * s + 1;
    if (s < 2) return a * s * s * s - 5 * a * s * s + 8 * a * s - 4 * a;
    return 0;
}

template <typename T>
__device__ __forceinline__ T keys_combine(const T g[4], const T k[4])
{
    return g[0] * k[0] + g[1] * k[1] + g[2] * k[2] + g[3] * k[3];
}

// Previous mesh displacement (X, Y) at (xi, eta): Keys bicubic with Keys' boundary
// extrapolation f(-1) = 3 f(0) - 3 f(1) + f(2) on Dirichlet grids, wrapped on periodic
// grids; or bilinear.
template <typename T>
__device__ void mesh_at(const McProblem<T>& P, T xi, T eta, T& ix, T& iy)
{
    int i, j;
    T tx, ty;
    locate(P.nx, P.periodic, xi, i, tx);
    locate(P.ny, P.periodic, eta, j, ty);
    const int nx = P.nx, ny = P.ny;
    const long N = (long)nx * ny;
    auto ld = [&](const Disp2<T>* q) { return load_disp(checked_ptr(q, P.disp, N)); };
    if (!P.bicubic) {
        const Disp2<T>* r0 = P.disp + (long)j * nx + i;
        const Disp2<T> a = ld(r0), b = ld(r0 + 1);
        const Disp2<T> c = ld(r0 + nx), d = ld(r0 + nx + 1);
        const T gx = 1 - tx, gy = 1 - ty;
        ix = gx * gy * a.X + tx * gy * b.X + gx * ty * c.X + tx * ty * d.X;
        iy = gx * gy * a.Y + tx * gy * b.Y + gx * ty * c.Y + tx * ty * d.Y;
        return;
    }
    const T kx[4] = {keys_kernel<T>(1 + tx), keys_kernel<T>(tx), keys_kernel<T>(1 - tx),
                     keys_kernel<T>(2 - tx)};
    const T ky[4] = {keys_kernel<T>(1 + ty), keys_kernel<T>(ty), keys_kernel<T>(1 - ty),
                     keys_kernel<T>(2 - ty)};
    T gX[4] = {0, 0, 0, 0}, gY[4] = {0, 0, 0, 0};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int r = j - 1 + b;
        if (P.periodic) {
            const int m = ny - 1;
            r = ((r % m) + m) % m;
        } else if (r < 0 || r > ny - 1) {
            continue;
        }
        const Disp2<T>* row = P.disp + (long)r * nx;
        T cX[4], cY[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int c = i - 1 + a;
            if (P.periodic) {
                const int m = nx - 1;
                c = ((c % m) + m) % m;
                const Disp2<T> v = ld(row + c);
                cX[a] = v.X;
                cY[a] = v.Y;
            } else if (c < 0) {
                const Disp2<T> v0 = ld(row), v1 = ld(row + 1), v2 = ld(row + 2);
                cX[a] = 3 * v0.X - 3 * v1.X + v2.X;
                cY[a] = 3 * v0.Y - 3 * v1.Y + v2.Y;
            } else if (c > nx - 1) {
                const Disp2<T> v0 = ld(row + nx - 1), v1 = ld(row + nx - 2), v2 = ld(row + nx - 3);
                cX[a] = 3 * v0.X - 3 * v1.X + v2.X;
                cY[a] = 3 * v0.Y - 3 * v1.Y + v2.Y;
            } else {
                const Disp2<T> v = ld(row + c);
                cX[a] = v.X;
                cY[a] = v.Y;
            }
        }
        gX[b] = keys_combine(cX, kx);
        gY[b] = keys_combine(cY, kx);
    }
    if (!P.periodic) {
        if (j - 1 < 0) {
            gX[0] = 3 * gX[1] - 3 * gX[2] + gX[3];
            gY[0] = 3 * gY[1] - 3 * gY[2] + gY[3];
        }
        if (j + 2 > ny - 1) {
            gX[3] = 3 * gX[2] - 3 * gX[1] + gX[0];
            gY[3] = 3 * gY[2] - 3 * gY[1] + gY[0];
        }
    }
    ix = keys_combine(gX, ky);
    iy = keys_combine(gY, ky);
}

template <typename T>
__device__ __forceinline__ T clamp01(T v) { return v < 0 ? (T)0 : (v > 1 ? (T)1 : v); }

// Linear interpolation along one side of the n boundary values b (nodes s = k / (n - 1)).
template <typename T>
__device__ __forceinline__ T side_lerp(const T* b, int n, T s)
{
    const T u = s * (T)(n - 1);
    int c = (int)dfloor(u);
    c = c < 0 ? 0 : (c > n - 2 ? n - 2 : c);
    const T f = u - (T)c;
    return ((T)1 - f) * b[checked(c, n)] + f * b[checked(c + 1, n)];
}

// Brownian-bridge crossing probability of one side, exp(-d0 d1 / (D ds)) with q = D ds; in FP64
// zero where the exponential is too small to change 1 - p (and then cannot be the largest p of
// an exiting path), which skips the exponential there.  One object per substep holds what the
// four sides share.
template <typename T> struct BridgeP {
    T q, lim;
    __device__ __forceinline__ explicit BridgeP(T q_)
    {
        q = q_;
        lim = Consts<T>::bridge_skip * q_;
    }
    __device__ __forceinline__ T operator()(T d0, T d1) const
    {
        const T a = d0 * d1;
        return (a > lim) ? (T)0 : dexp(-a / q);
    }
};
// FP32: the probability is only compared with a uniform deviate, so the hardware 2^x of
// a (-log2 e / q) serves (a few ulp), with the approximate division done once per substep rather
// than once per side.  No skip is needed: where a > 20 q, p < 2^-28.8, so 1 - p rounds to 1
// and such a side can never hold the largest p of an exiting path; 2^x of a large negative
// argument is 0.
template <> struct BridgeP<float> {
    float sc;
    __device__ __forceinline__ explicit BridgeP(float q_) { sc = __fdividef(-1.4426950408889634f, q_); }
    __device__ __forceinline__ float operator()(float d0, float d1) const
    {
        float r;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d0 * d1 * sc));
        return r;
    }
};

// Exit of a path whose proposed point (xn, en) left the unit square or whose bridge crossed side
// s (s < 0: the endpoint test fired; the side is the deepest violation, ties to the lower
// index): the exit point keeps the other coordinate of (xn, en), clamped to [0, 1], and the value
// is the boundary mesh there (the new boundary mesh along the side with a moving boundary).
// Returns the side.
template <typename T>
__device__ __forceinline__ int exit_value(const McProblem<T>& P, T xn, T en, int s, T& vx, T& vy)
{
    if (s < 0) {  // deepest violation
        T vmax = -xn;
        s = 0;
        if (xn - 1 > vmax) { vmax = xn - 1; s = 1; }
        if (-en > vmax) { vmax = -en; s = 2; }
        if (en - 1 > vmax) { vmax = en - 1; s = 3; }
    }
    T xe = clamp01(xn), ee = clamp01(en);
    if (s == 0) xe = 0;
    if (s == 1) xe = 1;
    if (s == 2) ee = 0;
    if (s == 3) ee = 1;
    if (P.bnd) {  // moving boundary: the new boundary mesh along the exit side
        if (s == 0) { vx = (T)0; vy = side_lerp(P.bnd + 2 * P.nx, P.ny, ee); }
        else if (s == 1) { vx = P.Lx; vy = side_lerp(P.bnd + 2 * P.nx + P.ny, P.ny, ee); }
        else if (s == 2) { vx = side_lerp(P.bnd, P.nx, xe); vy = (T)0; }
        else { vx = side_lerp(P.bnd + P.nx, P.nx, xe); vy = P.Ly; }
    } else {
        vx = P.Lx * xe;
        vy = P.Ly * ee;
    }
    return s;
}

// One substep k of path p at node m.  Returns 0 while the path goes on; 1 when it exits at this
// substep ((vx, vy) = the proposed point outside the square or across the bridge, side = the
// bridge's side or -1; exit_value turns them into the exit point and value later, for 32 exits at
// once); 2 when it completes its K-th substep ((xi, eta) = final point; its value, the previous
// mesh there, is evaluated later for 32 such paths at once).
// RK: the problem record holds the round keys in the launch's parameter block (single-problem
// launches); otherwise the keys are stepped inside the generator.
// The parts of Philox rounds 0 and 1 that do not depend on the substep k (counter (k, p, m, n)):
// round 0's product of word 2 (the node id m) and round 1's product of word 0 (which depends on
// p and m only) are taken once per path.
struct PhiloxHoist {
    uint32_t tz;    // n ^ rk1: round 0's word 2 input besides hi(M0 k)
    uint32_t y1k;   // lo(M1 m) ^ rk2: round 1's word 0 input besides hi(M1 z1)
    uint32_t H, L;  // hi, lo of M0 x1 with x1 = hi(M1 m) ^ p ^ rk0 (per path)
};

__device__ __forceinline__ U4 philox_hoisted(const uint32_t* rk, const PhiloxHoist& h, uint32_t k)
{
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    const uint32_t h0 = __umulhi(kM0, k), l0 = kM0 * k;
    const uint32_t z1 = h0 ^ h.tz;           // round 0 output (x1, y1, z1, l0)
    const uint32_t h1 = __umulhi(kM1, z1), l1 = kM1 * z1;
    U4 c{h1 ^ h.y1k, l1, h.H ^ l0 ^ rk[3], h.L};
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint32_t a0 = __umulhi(kM0, c.x), b0 = kM0 * c.x;
        const uint32_t a1 = __umulhi(kM1, c.z), b1 = kM1 * c.z;
        c = U4{a1 ^ c.y ^ rk[2 * r], b1, a0 ^ c.w ^ rk[2 * r + 1], b0};
    }
    return c;
}

template <typename T, bool RK>
__device__ __forceinline__ int path_substep(const McProblem<T>& P, uint32_t m, uint32_t p, int k,
                                             T& xi, T& eta, T& vx, T& vy, int& side, const PhiloxHoist& ph)
{
    // the monitor gather first: its loads are in flight while Philox runs
    T wv, wx, we;
    monitor_at(P, xi, eta, wv, wx, we);
    const U4 c{(uint32_t)k, p, m, P.tstep};
    U4 w;
    if constexpr (RK) w = philox_hoisted(P.rk, ph, (uint32_t)k);
    else w = philox4x32_10(c, P.key0, P.key1);
    const T u1 = uniform_open(w.x, T()), u2 = uniform_open(w.y, T()), ub = uniform_open(w.z, T());
    const T lgu = dlog(u1);
    T sn, cs;
    if constexpr (sizeof(T) == 4)
        sincos_2pi(u2, &sn, &cs);  // FP32: polynomial form (below 0.75 ulp)
    else
        sincos(Consts<T>::two_pi * u2, &sn, &cs);
    T q, bx, by;  // q = D ds, (bx, by) = drift * ds
    if (P.form == 0) {
        q = wv * P.cb;
        bx = wx * P.cb;
        by = we * P.cb;
    } else {
        q = P.cb;
        bx = wx / wv * P.cb;
        by = we / wv * P.cb;
    }
    // Eq. 7: increment sqrt(2 q) z with the Box-Muller normals z = sqrt(-2 ln u1) (cos, sin)(2 pi u2),
    // in the oracle's order of operations
    const T r = dsqrt((T)-2 * lgu);
    const T sd = dsqrt(2 * q);
    const T xn = xi + bx + sd * (r * cs);
    const T en = eta + by + sd * (r * sn);

    if (!P.periodic) {
        // outside the unit square: the largest violation is positive, i.e. the smallest of the
        // distances xn, 1 - xn, en, 1 - en is negative (1 - v is exactly -(v - 1) in floating
        // point, so the two forms decide alike); the distances serve the bridge test as well.
        // The side (ties keep the lower index) is found only for the paths that exit this way,
        // in the exit block.
        const T oxn = 1 - xn, oen = 1 - en;
        bool exited = dmin(dmin(xn, oxn), dmin(en, oen)) < 0;
        int s = -1;
        if (!exited && P.bb) {
            const BridgeP<T> bridge_p(q);
            const T p0 = bridge_p(xi, xn), p1 = bridge_p(1 - xi, oxn);
            const T p2 = bridge_p(eta, en), p3 = bridge_p(1 - eta, oen);
            T surv = 1;
            surv *= (1 - p0);
            surv *= (1 - p1);
            surv *= (1 - p2);
            surv *= (1 - p3);
            if (ub > surv) {
                exited = true;
                T pm = p0;
                s = 0;
                if (p1 > pm) { pm = p1; s = 1; }
                if (p2 > pm) { pm = p2; s = 2; }
                if (p3 > pm) { pm = p3; s = 3; }
            }
        }
        if (exited) {
            // the exit point, its value and its sums are formed later, for 32 exits at a time
            // (exit_value): here only the proposed point and the bridge side (-1: endpoint test)
            vx = xn;
            vy = en;
            side = s;
            return 1;
        }
    }
    xi = xn;
    eta = en;
    return k + 1 == P.K ? 2 : 0;
}

// Per-lane estimator sums of the shifted path values (shift = the node's previous position).
template <typename T, int ACC> struct LaneAcc;
template <typename T> struct LaneAcc<T, kAcc64> {
    double sx, sy;
    double s1x = 0, s2x = 0, s1y = 0, s2y = 0;
    __device__ __forceinline__ LaneAcc(double sx_, double sy_) : sx(sx_), sy(sy_) {}
    __device__ __forceinline__ void add(T vx, T vy)
    {
        const double dx = (double)vx - sx, dy = (double)vy - sy;
        s1x += dx;
        s2x += dx * dx;
        s1y += dy;
        s2y += dy * dy;
    }
    __device__ __forceinline__ void finish(double& a, double& b, double& c, double& d, unsigned long long, double,
                                           double) const
    {
        a = s1x; b = s2x; c = s1y; d = s2y;
    }
};
// Kahan-compensated FP32 sums of v - fl(shift): no FP64 work per path; converted to sums of
// v - shift (exact shift) once per task.  The x and y components run as paired FP32
// instructions, element for element the scalar operations (bit-identical sums).
template <typename T> struct LaneAcc<T, kAccKahan32> {
    float2 nshift;  // -fl(shift), (x, y)
    float2 s1 = {0.f, 0.f}, c1 = {0.f, 0.f}, s2 = {0.f, 0.f}, c2 = {0.f, 0.f};
    __device__ __forceinline__ LaneAcc(double sx, double sy) : nshift(make_float2(-(float)sx, -(float)sy)) {}
    __device__ __forceinline__ static float2 neg(float2 v) { return make_float2(-v.x, -v.y); }
    __device__ __forceinline__ static void kahan(float2& s, float2& c, float2 v)
    {
        const float2 y = __fadd2_rn(v, neg(c));
        const float2 t = __fadd2_rn(s, y);
        c = __fadd2_rn(__fadd2_rn(t, neg(s)), neg(y));
        s = t;
    }
    __device__ __forceinline__ void add(T vx, T vy)
    {
        const float2 d = __fadd2_rn(make_float2((float)vx, (float)vy), nshift);
        kahan(s1, c1, d);
        kahan(s2, c2, __fmul2_rn(d, d));
    }
    // sx, sy: the shifts again (read at the end of the task, so that they hold no registers while
    // paths run)
    __device__ __forceinline__ void finish(double& a, double& b, double& c, double& d, unsigned long long n,
                                           double sx, double sy) const
    {
        const double ex = sx - (double)(float)sx, ey = sy - (double)(float)sy;  // shift - fl(shift)
        const double S1x = (double)s1.x - (double)c1.x, S2x = (double)s2.x - (double)c2.x;
        const double S1y = (double)s1.y - (double)c1.y, S2y = (double)s2.y - (double)c2.y;
        const double nn = (double)n;
        a = S1x - nn * ex;
        b = S2x - 2.0 * ex * S1x + nn * ex * ex;
        c = S1y - nn * ey;
        d = S2y - 2.0 * ey * S1y + nn * ey * ey;
    }
};

// Paths pb .. pe-1 of local node m of problem R (global node g): one warp, one task.
// Per-warp shared-memory queues of ended paths: survivors (final point) wait for their bicubic
// terminal value, exits (proposed point and bridge side) for their boundary value; each is
// evaluated 32 at a time, one path per lane.
template <typename T> struct PathQueues {
    T* s_xi; T* s_eta; uint32_t* s_path;               // survivors
    T* e_xn; T* e_en; int32_t* e_side; int32_t* e_k; uint32_t* e_path;  // exits (k, path: debug)
};

template <typename T, int ACC, bool DEBUG, bool RK>
__device__ __forceinline__ void run_task(const McParams<T>& P, const McProblem<T>& R, int m, int g,
                                         int task, int64_t pb, int64_t pe, const PathQueues<T>& Q)
{
    T* q_xi = Q.s_xi;
    T* q_eta = Q.s_eta;
    uint32_t* q_path = Q.s_path;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int2 ij = R.nodes[m];
    const T xi0 = (T)ij.x / (T)(R.nx - 1);
    const T eta0 = (T)ij.y / (T)(R.ny - 1);
    const double sx = P.shift[2 * g], sy = P.shift[2 * g + 1];

    LaneAcc<T, ACC> acc(sx, sy);
    uint32_t steps = 0, paths = 0;          // per lane and task: far below 2^32
    uint32_t path = (uint32_t)pb + lane;    // path indices are below 2^32
    PhiloxHoist ph{};
    uint32_t x1base = 0;
    if constexpr (RK) {
        constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
        ph.tz = R.tstep ^ R.rk[1];
        ph.y1k = (kM1 * (uint32_t)m) ^ R.rk[2];
        x1base = __umulhi(kM1, (uint32_t)m) ^ R.rk[0];
        const uint32_t x1 = x1base ^ path;
        ph.H = __umulhi(kM0, x1);
        ph.L = kM0 * x1;
    }
    const uint32_t pend = (uint32_t)pe;
    bool live = path < pend;
    uint32_t next = (uint32_t)pb + 32;
    T xi = xi0, eta = eta0;
    int k = 0;
    int qn = 0;  // completed paths waiting for their terminal value (warp-uniform)
    // terminal values of `count` queued paths at once, one per lane
    auto drain = [&](int count) {
        __syncwarp();
        if (lane < count) {
            const int pos = checked(qn - count + lane, 64);
            const T fx = q_xi[pos], fy = q_eta[pos];
            T ix, iy;
            mesh_at(R, fx, fy, ix, iy);
            const T vx = R.Lx * fx + ix, vy = R.Ly * fy + iy;
            acc.add(vx, vy);
            if (DEBUG) {
                const int64_t qd = (int64_t)q_path[pos] - P.dbg_p0;  // debug only
                P.dbg_val[2 * qd] = (double)vx;
                P.dbg_val[2 * qd + 1] = (double)vy;
                P.dbg_steps[qd] = R.K;
                P.dbg_side[qd] = (int8_t)4;
            }
        }
        qn -= count;
        __syncwarp();
    };
    int qe = 0;  // exited paths waiting for their boundary value (warp-uniform)
    auto drain_exits = [&](int count) {
        __syncwarp();
        if (lane < count) {
            const int pos = checked(qe - count + lane, 64);
            T vx, vy;
            const int side = exit_value(R, Q.e_xn[pos], Q.e_en[pos], (int)Q.e_side[pos], vx, vy);
            acc.add(vx, vy);
            if (DEBUG) {
                const int64_t qd = (int64_t)Q.e_path[pos] - P.dbg_p0;  // debug only
                P.dbg_val[2 * qd] = (double)vx;
                P.dbg_val[2 * qd + 1] = (double)vy;
                P.dbg_steps[qd] = Q.e_k[pos];
                P.dbg_side[qd] = (int8_t)side;
            }
        }
        qe -= count;
        __syncwarp();
    };
    while (__any_sync(kFull, live)) {
        int st = 0;
        T vx, vy;
        int side = 0;
        if (live) {
            st = path_substep<T, RK>(R, (uint32_t)m, path, k, xi, eta, vx, vy, side, ph);
            ++k;
            if (st != 0) {
                steps += (uint32_t)k;
                paths += 1;
            }
        }
        const unsigned dm = __ballot_sync(kFull, st != 0);
        if (dm) {  // some lane's path ended: queue survivors (and exits), hand out the next path indices
            const unsigned sm = __ballot_sync(kFull, st == 2);
            if (st == 2) {
                const int pos = checked(qn + __popc(sm & lt), 64);
                q_xi[pos] = xi;
                q_eta[pos] = eta;
                if (DEBUG) q_path[pos] = path;
            }
            qn += __popc(sm);
            const unsigned em = dm & ~sm;  // exits
            if (st == 1) {
                const int pos = checked(qe + __popc(em & lt), 64);
                Q.e_xn[pos] = vx;
                Q.e_en[pos] = vy;
                Q.e_side[pos] = side;
                if (DEBUG) {
                    Q.e_k[pos] = k;
                    Q.e_path[pos] = path;
                }
            }
            qe += __popc(em);
            if (st != 0) {
                path = next + __popc(dm & lt);
                if constexpr (RK) {
                    const uint32_t x1 = x1base ^ path;
                    ph.H = __umulhi(0xD2511F53u, x1);
                    ph.L = 0xD2511F53u * x1;
                }
                live = path < pend;
                xi = xi0;
                eta = eta0;
                k = 0;
            }
            next += __popc(dm);
            if (qn >= 32) drain(32);
            if (qe >= 32) drain_exits(32);
        }
    }
    if (qn > 0) drain(qn);
    if (qe > 0) drain_exits(qe);
    double a, b, c, d;
    acc.finish(a, b, c, d, paths, P.shift[2 * g], P.shift[2 * g + 1]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(kFull, a, off);
        b += __shfl_xor_sync(kFull, b, off);
        c += __shfl_xor_sync(kFull, c, off);
        d += __shfl_xor_sync(kFull, d, off);
        steps += __shfl_xor_sync(kFull, steps, off);
        paths += __shfl_xor_sync(kFull, paths, off);
    }
    if (lane == 0) P.slots[task] = TaskSlot{a, b, c, d, steps, paths};
}

// Persistent path kernel.  BATCH: tasks of several problems share the launch; each task reads
// its problem's record (the Philox counter uses the problem-local node id, so a problem's
// results do not depend on what else shares the launch).
template <typename T, int ACC, bool DEBUG, bool BATCH, int TPB = kMcThreads>
__global__ void __launch_bounds__(TPB, (mc_min_blocks<T, TPB>())) mc_kernel(const __grid_constant__ McParams<T> P)
{
    constexpr int kWarps = TPB / 32;
    constexpr int kD = DEBUG ? 64 : 1;  // debug-only entries per warp
    __shared__ T q_xi[kWarps][64], q_eta[kWarps][64];
    __shared__ uint32_t q_path[kWarps][kD];
    __shared__ T e_xn[kWarps][64], e_en[kWarps][64];
    __shared__ int32_t e_side[kWarps][64];
    __shared__ int32_t e_k[kWarps][kD];
    __shared__ uint32_t e_path[kWarps][kD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const PathQueues<T> Q{q_xi[warp], q_eta[warp], q_path[warp], e_xn[warp], e_en[warp], e_side[warp], e_k[warp],
                          e_path[warp]};
    const int n_active = *P.n_active;
    const int64_t n_tasks = P.task_off[n_active];
    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(P.task_counter, 1);
        task = __shfl_sync(kFull, task, 0);
        if ((int64_t)task >= n_tasks) break;
        int lo = 0, hi = n_active - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.task_off[mid] <= task) lo = mid; else hi = mid - 1;
        }
        const int g = P.node_of[lo];
        const int64_t chunk_end = P.p_begin[lo] + P.p_count[lo];
        const int64_t tp = P.task_paths > 0 ? P.task_paths : kPathsPerTask;
        const int64_t pb = P.p_begin[lo] + ((int64_t)task - P.task_off[lo]) * tp;
        const int64_t pe = pb + tp < chunk_end ? pb + tp : chunk_end;
        if constexpr (BATCH) {
            const McProblem<T> R = P.probs[P.node_prob[g]];
            run_task<T, ACC, DEBUG, false>(P, R, g - R.node_offset, g, task, pb, pe, Q);
        } else {
            run_task<T, ACC, DEBUG, true>(P, P.prob, g, g, task, pb, pe, Q);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Round plan: compact the nodes that still need paths, cut their chunks into tasks.
// One block; node order is preserved so the plan is deterministic.
// ---------------------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;

template <typename V>
__device__ V block_exclusive_scan(V v, V* warp_tot, V& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const V o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        V t = lane < nw ? warp_tot[lane] : (V)0;
        V ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const V o = __shfl_up_sync(kFull, ti, off);
            if (lane >= off) ti += o;
        }
        if (lane < nw) warp_tot[lane] = ti - t;   // exclusive prefix of warp totals
        if (lane == nw - 1) warp_tot[32] = ti;    // block total
    }
    __syncthreads();
    const V res = warp_tot[wid] + incl - v;
    total = warp_tot[32];
    __syncthreads();
    return res;
}

// Node of planning position v: v itself, or (ranges given) position v of the concatenation of
// the ranges [range_off[r], range_off[r] + range_pre[r+1] - range_pre[r]) in list order.
__device__ __forceinline__ int plan_node(const PlanParams& P, int v)
{
    if (!P.range_off) return v;
    int lo = 0, hi = P.n_ranges - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.range_pre[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return P.range_off[lo] + (v - P.range_pre[lo]);
}

// With max_tasks > 0 the round takes nodes in planning order while the tasks before them number
// fewer than max_tasks (at least the first pending node); later nodes keep their chunk for a
// later round.  A node's chunks, and hence its results, do not depend on the cap.
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(const PlanParams P)
{
    __shared__ int64_t s_tasks[33];
    __shared__ int s_act[33];
    const int64_t tp = P.task_paths > 0 ? P.task_paths : kPathsPerTask;
    const int64_t max_chunk = (int64_t)kTasksPerRound * tp;  // 2^19 paths at the default task size
    int64_t task_base = 0;
    int act_base = 0;
    for (int base = 0; base < P.M; base += kPlanThreads) {
        const int v = base + threadIdx.x;
        const int m = v < P.M ? plan_node(P, v) : 0;
        int64_t cnt = 0;
        if (v < P.M) {
            cnt = P.next_total[m] - P.n_done[m];
            if (cnt > max_chunk) cnt = max_chunk;
            if (cnt < 0) cnt = 0;
        }
        const int64_t tasks = cnt > 0 ? (cnt + tp - 1) / tp : 0;
        int64_t task_tot;
        const int64_t t_ex = block_exclusive_scan<int64_t>(tasks, s_tasks, task_tot);
        // the cap excludes a suffix of this block's nodes, so t_ex is also the prefix over the
        // nodes that stay
        const bool fits = P.max_tasks <= 0 || task_base + t_ex < P.max_tasks;
        const int act = (cnt > 0 && fits) ? 1 : 0;
        int act_tot;
        const int a_ex = block_exclusive_scan<int>(act, s_act, act_tot);
        int64_t kept_tot;
        (void)block_exclusive_scan<int64_t>(act ? tasks : 0, s_tasks, kept_tot);
        if (act) {
            const int a = act_base + a_ex;
            P.node_of[a] = m;
            P.p_begin[a] = P.n_done[m];
            P.p_count[a] = cnt;
            P.task_off[a] = task_base + t_ex;
        }
        act_base += act_tot;
        task_base += kept_tot;
        if (P.max_tasks > 0 && task_base >= P.max_tasks) break;
    }
    if (threadIdx.x == 0) {
        P.task_off[act_base] = task_base;
        *P.n_active = act_base;
        *P.task_counter = 0;
    }
}

__global__ void mc_init_kernel(int M, int64_t n0, int64_t max_paths, double* acc, int64_t* n_done,
                               int64_t* steps, int64_t* paths_run, int64_t* next_total, const int32_t* role)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    acc[4 * m] = acc[4 * m + 1] = acc[4 * m + 2] = acc[4 * m + 3] = 0.0;
    n_done[m] = 0;
    steps[m] = 0;
    paths_run[m] = 0;
    const bool interpolated = role && role[m] >= 0;
    next_total[m] = interpolated ? 0 : (n0 < max_paths ? n0 : max_paths);
}

// Interface sampling (Sec. 3.6): interpolated nodes from the estimates of their anchors, in the
// order w va + (1 - w) vb without fused multiply-add; their standard error is 0.
__global__ void interp_kernel(const InterpRule* rules, int n, double* est, double* se)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const InterpRule r = rules[k];
    const double ax = __dadd_rn(r.a >= 0 ? est[2 * r.a] : 0.0, r.oax);
    const double ay = __dadd_rn(r.a >= 0 ? est[2 * r.a + 1] : 0.0, r.oay);
    const double bx = __dadd_rn(r.b >= 0 ? est[2 * r.b] : 0.0, r.obx);
    const double by = __dadd_rn(r.b >= 0 ? est[2 * r.b + 1] : 0.0, r.oby);
    const double wb = __dsub_rn(1.0, r.w);
    est[2 * r.m] = __dadd_rn(__dmul_rn(r.w, ax), __dmul_rn(wb, bx));
    est[2 * r.m + 1] = __dadd_rn(__dmul_rn(r.w, ay), __dmul_rn(wb, by));
    se[2 * r.m] = 0.0;
    se[2 * r.m + 1] = 0.0;
}

__device__ __forceinline__ void node_estimate(const double* s, double n, double sx, double sy,
                                              double& mx, double& my, double& ex, double& ey)
{
    mx = sx + s[0] / n;
    my = sy + s[2] / n;
    double vx = (s[1] - s[0] * s[0] / n) / (n - 1.0);
    double vy = (s[3] - s[2] * s[2] / n) / (n - 1.0);
    vx = vx > 0 ? vx : 0.0;
    vy = vy > 0 ? vy : 0.0;
    ex = sqrt(vx / n);
    ey = sqrt(vy / n);
}

// One warp per active node: add its task slots in task order to the node's sums, then
// schedule its next total (adaptive mode).
__global__ void reduce_kernel(const ReduceParams P)
{
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= *P.n_active) return;
    const int m = P.node_of[a];
    const int64_t t0 = P.task_off[a], t1 = P.task_off[a + 1];
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    unsigned long long st = 0, np = 0;
    for (int64_t t = t0 + lane; t < t1; t += 32) {
        const TaskSlot v = P.slots[t];
        s0 += v.s1x; s1 += v.s2x; s2 += v.s1y; s3 += v.s2y;
        st += v.steps; np += v.paths;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(kFull, s0, off);
        s1 += __shfl_xor_sync(kFull, s1, off);
        s2 += __shfl_xor_sync(kFull, s2, off);
        s3 += __shfl_xor_sync(kFull, s3, off);
        st += __shfl_xor_sync(kFull, st, off);
        np += __shfl_xor_sync(kFull, np, off);
    }
    if (lane != 0) return;
    double* s = P.acc + 4 * m;
    s[0] += s0; s[1] += s1; s[2] += s2; s[3] += s3;
    P.steps[m] += (int64_t)st;
    P.paths_run[m] += (int64_t)np;
    const int64_t n = P.n_done[m] + P.p_count[a];
    P.n_done[m] = n;
    if (n < P.next_total[m]) return;  // chunk capped by the round size: keep the schedule
    if (P.se_target > 0) {
        double mx, my, ex, ey;
        node_estimate(s, (double)n, P.shift[2 * m], P.shift[2 * m + 1], mx, my, ex, ey);
        P.next_total[m] = adaptive_next_total(n, ex > ey ? ex : ey, P.se_target, P.max_paths);
    } else {
        P.next_total[m] = n;
    }
}

__global__ void output_kernel(int M, const double* acc, const int64_t* n_done, const double* shift,
                              double* est, double* se)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double mx, my, ex, ey;
    node_estimate(acc + 4 * m, (double)n_done[m], shift[2 * m], shift[2 * m + 1], mx, my, ex, ey);
    est[2 * m] = mx;
    est[2 * m + 1] = my;
    se[2 * m] = ex;
    se[2 * m + 1] = ey;
}

__global__ void philox_kernel(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 r = philox4x32_10(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]},
                               key[2 * i], key[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

template <typename T, int ACC, bool DEBUG, bool BATCH, int TPB = kMcThreads>
const void* mc_kernel_ptr()
{
    return reinterpret_cast<const void*>(&mc_kernel<T, ACC, DEBUG, BATCH, TPB>);
}

template <typename T, int TPB>
const void* select_batch_mc(int acc_mode)
{
    return acc_mode == kAccKahan32 ? mc_kernel_ptr<T, kAccKahan32, false, true, TPB>()
                                   : mc_kernel_ptr<T, kAcc64, false, true, TPB>();
}

template <typename T>
const void* select_mc(int acc_mode, bool debug, bool batch, int tpb)
{
    if (batch) {
        if (tpb == 128) return select_batch_mc<T, 128>(acc_mode);
        if (tpb == 512) return select_batch_mc<T, 512>(acc_mode);
        return select_batch_mc<T, kMcThreads>(acc_mode);
    }
    if (debug) return acc_mode == kAccKahan32 ? mc_kernel_ptr<T, kAccKahan32, true, false>()
                                              : mc_kernel_ptr<T, kAcc64, true, false>();
    return acc_mode == kAccKahan32 ? mc_kernel_ptr<T, kAccKahan32, false, false>()
                                   : mc_kernel_ptr<T, kAcc64, false, false>();
}

}  // namespace

template <typename T, int TPB>
void launch_batch_mc_kernel(const McParams<T>& P, bool kahan, int grid, cudaStream_t s)
{
    if (kahan) mc_kernel<T, kAccKahan32, false, true, TPB><<<grid, TPB, 0, s>>>(P);
    else mc_kernel<T, kAcc64, false, true, TPB><<<grid, TPB, 0, s>>>(P);
}

template <typename T>
cudaError_t launch_mc(const McParams<T>& P, int acc_mode, bool debug, bool batch, int grid, cudaStream_t s,
                      int tpb)
{
    const bool kahan = acc_mode == kAccKahan32;
    if (batch) {
        if (tpb == 128) launch_batch_mc_kernel<T, 128>(P, kahan, grid, s);
        else if (tpb == 512) launch_batch_mc_kernel<T, 512>(P, kahan, grid, s);
        else launch_batch_mc_kernel<T, kMcThreads>(P, kahan, grid, s);
    } else if (debug) {
        if (kahan) mc_kernel<T, kAccKahan32, true, false><<<grid, kMcThreads, 0, s>>>(P);
        else mc_kernel<T, kAcc64, true, false><<<grid, kMcThreads, 0, s>>>(P);
    } else {
        if (kahan) mc_kernel<T, kAccKahan32, false, false><<<grid, kMcThreads, 0, s>>>(P);
        else mc_kernel<T, kAcc64, false, false><<<grid, kMcThreads, 0, s>>>(P);
    }
    return cudaGetLastError();
}

template <typename T>
int mc_max_blocks_per_sm(int acc_mode, bool debug, bool batch, int tpb)
{
    int nb = 0;
    const int threads = batch && (tpb == 128 || tpb == 512) ? tpb : kMcThreads;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, select_mc<T>(acc_mode, debug, batch, tpb), threads,
                                                      0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template cudaError_t launch_mc<float>(const McParams<float>&, int, bool, bool, int, cudaStream_t, int);
template cudaError_t launch_mc<double>(const McParams<double>&, int, bool, bool, int, cudaStream_t, int);
template int mc_max_blocks_per_sm<float>(int, bool, bool, int);
template int mc_max_blocks_per_sm<double>(int, bool, bool, int);

cudaError_t launch_mc_init(int M, int64_t n0, int64_t max_paths, double* acc, int64_t* n_done,
                           int64_t* steps, int64_t* paths_run, int64_t* next_total, cudaStream_t s,
                           const int32_t* role)
{
    mc_init_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, n0, max_paths, acc, n_done, steps, paths_run,
                                                   next_total, role);
    return cudaGetLastError();
}

cudaError_t launch_interp(const InterpRule* rules, int n, double* est, double* se, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    interp_kernel<<<(n + 255) / 256, 256, 0, s>>>(rules, n, est, se);
    return cudaGetLastError();
}

cudaError_t launch_plan(const PlanParams& P, cudaStream_t s)
{
    plan_kernel<<<1, kPlanThreads, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceParams& P, int M, cudaStream_t s)
{
    const int threads = 256;
    const long warps = M;
    reduce_kernel<<<(int)((warps * 32 + threads - 1) / threads), threads, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_output(int M, const double* acc, const int64_t* n_done, const double* shift,
                          double* est, double* se, cudaStream_t s)
{
    output_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, acc, n_done, shift, est, se);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                          cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, key, n, out);
    return cudaGetLastError();
}

}  // namespace sdd

extern "C" int64_t sdd_debug_bounds_violations(void)
{
#ifdef SDD_BOUNDS_CHECK
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -2;
    if (cudaMemcpyFromSymbol(&v, sdd::g_bounds_violations, sizeof v) != cudaSuccess) return -2;
    return (int64_t)v;
#else
    return -1;
#endif
}
