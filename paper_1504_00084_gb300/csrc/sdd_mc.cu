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
// (k, p, m, n) -> Box-Muller normals (words 0, 1; FP32: log_unit, sqrt_pos2, sincos_2pi) and
// the bridge uniform (word 2); bilinear gather of {omega, omega_xi, omega_eta} from the packed
// monitor (read-only cache; FP32: one 64-byte cell record of the four corners, two 32-byte
// loads; FP64: four 32-byte node records); Euler-Maruyama update (Eq. 7); endpoint and
// Brownian-bridge exit tests.  Terminal values: the boundary mesh at
// the exit point, or the Keys-bicubic previous mesh at the final point (Eq. 5a, Eq. 6).
//
// Reductions: per-lane sums of the shifted values (FP64, or Kahan-compensated FP32), a
// fixed xor-shuffle tree per task, one slot per task, then one warp per node adds its slots
// in task order.  No floating-point atomics: results are bitwise reproducible.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

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
    // the sine (x) and cosine (y) series side by side, one paired instruction per degree:
    // coefficients (pi/2)^9/9!, -(pi/2)^10/10! down to pi/2, -(pi/2)^2/2!; then x r and y r2 + 1
    float2 pp = __ffma2_rn(make_float2(0x1.507834p-13f, -0x1.a6d1f2p-16f), make_float2(r2, r2),
                           make_float2(-0x1.32d2ccp-8f, 0x1.e1f506p-11f));
    pp = __ffma2_rn(pp, make_float2(r2, r2), make_float2(0x1.466bc6p-4f, -0x1.55d3c8p-6f));
    pp = __ffma2_rn(pp, make_float2(r2, r2), make_float2(-0x1.4abbcep-1f, 0x1.03c1f0p-2f));
    pp = __ffma2_rn(pp, make_float2(r2, r2), make_float2(0x1.921fb6p+0f, -0x1.3bd3ccp+0f));
    pp = __ffma2_rn(pp, make_float2(r, r2), make_float2(0.0f, 1.0f));
    // quadrant q mod 4: odd quadrants swap sine and cosine; the sine is negative in quadrants
    // 2, 3 (bit 1 of q), the cosine in quadrants 1, 2 (bit 1 of q + 1): set as the sign bit
    const bool odd = qint & 1;
    const float s_ = odd ? pp.y : pp.x;
    const float c_ = odd ? pp.x : pp.y;
    *sn = __int_as_float(__float_as_int(s_) ^ ((uint32_t)qint << 30 & 0x80000000u));
    *cs = __int_as_float(__float_as_int(c_) ^ ((uint32_t)(qint + 1) << 30 & 0x80000000u));
}

// Square roots of two positive normal FP32 numbers (here -2 ln u1 >= 1.2e-7 and 2 q > 0): the
// hardware reciprocal square root estimate r of a, then one Newton correction of y = a r,
// y + (a - y^2) r / 2, with the residual a - y^2 formed exactly by the fused multiply-add
// (Markstein's scheme for square roots).  The estimate's relative error near 2^-23 leaves the
// correction's error far below half an ulp, so the result is the rounded square root except
// where that lies within that error of a rounding boundary (checked against sqrtf over every
// float in [2^-24, 2^8]).  No zero, infinity, NaN or subnormal handling: the arguments exclude them.
__device__ __forceinline__ float2 sqrt_pos2(float2 a)
{
    float r0, r1;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(a.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(a.y));
    const float2 y = __fmul2_rn(a, make_float2(r0, r1));
    const float2 h = __fmul2_rn(make_float2(r0, r1), make_float2(0.5f, 0.5f));
    const float2 e = __ffma2_rn(make_float2(-y.x, -y.y), y, a);
    return __ffma2_rn(e, h, y);
}

// Natural logarithm of a uniform u in [2^-24, 1) (the FP32 deviates of uniform_open): with
// u = 2^e m, m in [sqrt(1/2), sqrt(2)) and f = m - 1 (exact), ln u = e ln 2 + ln(1 + f), and
// ln(1 + f) = f + f^2 P(f) with P the degree-8 polynomial fitted to (ln(1 + f) - f) / f^2 on that
// range (weighted least squares on Chebyshev nodes, coefficients rounded to FP32: fit_log_unit.py
// beside this file prints them); e ln 2 is added
// as e ln2_hi + (e ln2_lo + ...), ln2_hi = ln 2 rounded to FP32.  Checked over all 2^23 such
// uniforms against the rounded FP64 logarithm: within 1 ulp, rounded correctly for 93 % of them.
// No zero, negative, infinite or subnormal arguments (uniform_open makes none).
__device__ __forceinline__ float log_unit(float u)
{
    const int i = __float_as_int(u);
    const int e = (i - 0x3F3504F3) >> 23;                             // 0x3F3504F3: sqrt(1/2)
    const float f = __int_as_float(i - (int)((uint32_t)e << 23)) - 1.0f;
    const float ef = __int_as_float(e + 0x4B400000) - 0x1.8p23f;      // e, exactly
    float p = -0x1.3997c2p-4f;
    p = fmaf(p, f, 0x1.04605ep-3f);
    p = fmaf(p, f, -0x1.0ce6acp-3f);
    p = fmaf(p, f, 0x1.22f1e8p-3f);
    p = fmaf(p, f, -0x1.54830ap-3f);
    p = fmaf(p, f, 0x1.999fb8p-3f);
    p = fmaf(p, f, -0x1.00020cp-2f);
    p = fmaf(p, f, 0x1.555554p-2f);
    p = fmaf(p, f, -0x1.fffffep-2f);
    const float t = fmaf(f * f, p, f);
    return fmaf(ef, 0x1.62e430p-1f, fmaf(ef, -0x1.05c610p-29f, t));
}

template <typename T> struct Consts;
template <> struct Consts<double> {
    static constexpr double two_pi = 6.28318530717958647692;
    // exp(-a) below this argument's reach leaves 1 - exp(-a) == 1 exactly (and cannot be the
    // largest crossing probability of an exiting path), so the exponential is skipped.
    static constexpr double bridge_skip = 40.0;
};

// Two consecutive Mon4<float> records (32 bytes, 32-byte aligned) in one read-only 256-bit load.
__device__ __forceinline__ void ld_cell_half(const float* p, Mon4<float>& r0, Mon4<float>& r1)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r0.w), "=f"(r0.wx), "=f"(r0.we), "=f"(r0.pad), "=f"(r1.w), "=f"(r1.wx), "=f"(r1.we), "=f"(r1.pad)
        : "l"(p));
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

// Products and sums that no build fuses into a multiply-add: where the path's decisions follow
// the oracle's arithmetic operation for operation (the oracle itself is compiled without fused
// multiply-adds).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// The problem switches a substep reads: from the problem record (FL < 0), or fixed at compile
// time (FL >= 0: bit 0 periodic, bit 1 the paper's generator form, bit 2 the bridge test), so
// that the common configurations run without their per-substep branches.
template <int FL> struct Mode {
    template <typename T> __device__ __forceinline__ static bool periodic(const McProblem<T>& P)
    {
        if constexpr (FL < 0) return P.periodic != 0; else return (FL & 1) != 0;
    }
    template <typename T> __device__ __forceinline__ static bool form1(const McProblem<T>& P)
    {
        if constexpr (FL < 0) return P.form != 0; else return (FL & 2) != 0;
    }
    template <typename T> __device__ __forceinline__ static bool bridge(const McProblem<T>& P)
    {
        if constexpr (FL < 0) return P.bb != 0; else return (FL & 4) != 0;
    }
};
constexpr int kModeDirichletBridge = 4;       // Dirichlet, generator form tau x_t = div(w grad x)
constexpr int kModeDirichletBridgeForm1 = 6;  // Dirichlet, the paper's generator form

// Bilinear interpolation of the packed monitor at (xi, eta) (Sec. 3.4).
// FP32 Dirichlet grids locate the cell without conversions: for a coordinate s in [0, 1] on an
// n-node line, u = s (n - 1) + 2^23 rounded down holds floor(u) in its low mantissa bits (unit
// spacing there), so it is the float 2^23 + cell exactly, with bits 0x4B000000 + cell, and the
// offset u - cell is exact; s = 1 gives cell n - 1 with offset 0, whose clamped corner records
// carry zero weight.  The cell record j nx + i is then bits_j nx + bits_i - (nx + 1) 0x4B000000
// (mod 2^32).  Both coordinates run as paired FP32 instructions.  Paths inside the unit square
// only (a Dirichlet path leaves at its first step outside).
template <typename T, bool PARAM, int FL>
__device__ __forceinline__ void monitor_at(const McProblem<T>& P, T xi, T eta, T& w, T& wx, T& we)
{
    T fx, fy;
    int base;  // grids hold at most 2^28 nodes
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (!Mode<FL>::periodic(P)) {
            float2 u;
            if constexpr (PARAM)  // the record lives in the parameter block: its constants are operands
                u = __fmul2_rn(make_float2(xi, eta), make_float2(P.gs[0], P.gs[1]));
            else                  // a record in registers: convert rather than hold two more values
                u = __fmul2_rn(make_float2(xi, eta), make_float2((float)(P.nx - 1), (float)(P.ny - 1)));
            const float2 t = __fadd2_rd(u, make_float2(0x1.0p23f, 0x1.0p23f));
            const float2 c = __fadd2_rn(t, make_float2(-0x1.0p23f, -0x1.0p23f));  // the cells, exactly
            const float2 f = __ffma2_rn(c, make_float2(-1.0f, -1.0f), u);          // u - cell, exactly
            fx = f.x;
            fy = f.y;
            // the cell of a position in the unit square; any other value (a NaN from invalid input,
            // which the step reports afterwards) is held to the last record by one unsigned minimum
            base = (int)min((uint32_t)__float_as_int(t.y) * (uint32_t)P.nx + (uint32_t)__float_as_int(t.x) - P.cell_bias,
                            P.cell_last);
            done = true;
        }
    }
    if (!done) {
        int i, j;
        locate(P.nx, (int)Mode<FL>::periodic(P), xi, i, fx);
        locate(P.ny, (int)Mode<FL>::periodic(P), eta, j, fy);
        base = j * P.nx + i;  // FP32 cell record, FP64 node record
    }
    Mon4<T> a, b, c, d;
    if constexpr (sizeof(T) == 4) {  // the cell's four corner records: two 32-byte loads
        const long cells = (long)P.nx * P.ny;
        const float* q = reinterpret_cast<const float*>(P.mon) + 16 * (long)checked(base, cells);
        ld_cell_half(q, a, b);
        ld_cell_half(q + 8, c, d);
    } else {
        const long N = (long)P.nx * P.ny;
        a = load_mon(P.mon + checked(base, N));
        b = load_mon(P.mon + checked(base + 1, N));
        c = load_mon(P.mon + checked(base + P.nx, N));
        d = load_mon(P.mon + checked(base + P.nx + 1, N));
    }
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
        // w00 f00 + w10 f10 + w01 f01 + w11 f11 from the left, each operation rounded (as the oracle)
        const T gx = add_rn((T)1, -fx), gy = add_rn((T)1, -fy);
        const T w00 = mul_rn(gx, gy), w10 = mul_rn(fx, gy), w01 = mul_rn(gx, fy), w11 = mul_rn(fx, fy);
        auto bil = [&](T f00, T f10, T f01, T f11) {
            return add_rn(add_rn(add_rn(mul_rn(w00, f00), mul_rn(w10, f10)), mul_rn(w01, f01)), mul_rn(w11, f11));
        };
        w = bil(a.w, b.w, c.w, d.w);
        wx = bil(a.wx, b.wx, c.wx, d.wx);
        we = bil(a.we, b.we, c.we, d.we);
    }
}

// Keys (1981) cubic-convolution kernel, a = -1/2: 3/2 s^3 - 5/2 s^2 + 1 on [0, 1],
// -1/2 s^3 + 5/2 s^2 - 4 s + 2 on [1, 2], in Horner form.  The arithmetic here and below is
// written as explicit fused multiply-adds, so that every build and every kernel instantiation
// rounds alike (a batched problem then reproduces the same problem stepped alone bit for bit).
template <typename T>
__device__ __forceinline__ T keys_kernel(T s)
{
    s = dabs(s);
    if (s <= 1) return fma(fma((T)1.5, s, (T)-2.5), s * s, (T)1);
    if (s < 2) return fma(fma(fma((T)-0.5, s, (T)2.5), s, (T)-4), s, (T)2);
    return 0;
}

template <typename T>
__device__ __forceinline__ T keys_combine(const T g[4], const T k[4])
{
    return fma(g[3], k[3], fma(g[2], k[2], fma(g[1], k[1], g[0] * k[0])));
}

// Keys' boundary extrapolation 3 f0 - 3 f1 + f2.
template <typename T>
__device__ __forceinline__ T keys_extrap(T f0, T f1, T f2)
{
    return fma((T)3, f0, fma((T)-3, f1, f2));
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
        const T w00 = gx * gy, w10 = tx * gy, w01 = gx * ty, w11 = tx * ty;
        ix = fma(w11, d.X, fma(w01, c.X, fma(w00, a.X, w10 * b.X)));
        iy = fma(w11, d.Y, fma(w01, c.Y, fma(w00, a.Y, w10 * b.Y)));
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
                cX[a] = keys_extrap(v0.X, v1.X, v2.X);
                cY[a] = keys_extrap(v0.Y, v1.Y, v2.Y);
            } else if (c > nx - 1) {
                const Disp2<T> v0 = ld(row + nx - 1), v1 = ld(row + nx - 2), v2 = ld(row + nx - 3);
                cX[a] = keys_extrap(v0.X, v1.X, v2.X);
                cY[a] = keys_extrap(v0.Y, v1.Y, v2.Y);
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
            gX[0] = keys_extrap(gX[1], gX[2], gX[3]);
            gY[0] = keys_extrap(gY[1], gY[2], gY[3]);
        }
        if (j + 2 > ny - 1) {
            gX[3] = keys_extrap(gX[2], gX[1], gX[0]);
            gY[3] = keys_extrap(gY[2], gY[1], gY[0]);
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
    return fma(f, b[checked(c + 1, n)], ((T)1 - f) * b[checked(c, n)]);
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
        vx = mul_rn(P.Lx, xe);
        vy = mul_rn(P.Ly, ee);
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

template <typename T, bool RK, int FL>
__device__ __forceinline__ int path_substep(const McProblem<T>& P, uint32_t m, uint32_t p, int k,
                                             T& xi, T& eta, T& vx, T& vy, int& side, const PhiloxHoist& ph)
{
    // the monitor gather first: its loads are in flight while Philox runs
    T wv, wx, we;
    monitor_at<T, RK, FL>(P, xi, eta, wv, wx, we);
    const U4 c{(uint32_t)k, p, m, P.tstep};
    U4 w;
    if constexpr (RK) w = philox_hoisted(P.rk, ph, (uint32_t)k);
    else w = philox4x32_10(c, P.key0, P.key1);
    if constexpr (sizeof(T) == 4) {
        // FP32: the generic form's steps below, with the kernel's own logarithm, square roots and
        // sin/cos, the noise term of the update fused, and the x and y (and paired bridge-side)
        // work as paired FP32 instructions
        const float2 u12 = __fadd2_rn(make_float2(__int_as_float((w.x >> 9) + 0x3F800000u),
                                                  __int_as_float((w.y >> 9) + 0x3F800000u)),
                                      make_float2(-0x1.fffffep-1f, -0x1.fffffep-1f));
        const float ub = uniform_open(w.z, 0.0f);
        const float lgu = log_unit(u12.x);
        float sn, cs;
        sincos_2pi(u12.y, &sn, &cs);
        float q;
        float2 b;  // drift * ds, each product rounded as in the oracle (never fused into the add below)
        if (!Mode<FL>::form1(P)) {
            q = wv * P.cb;
            b = make_float2(__fmul_rn(wx, P.cb), __fmul_rn(we, P.cb));
        } else {
            q = P.cb;
            b = make_float2(__fmul_rn(wx / wv, P.cb), __fmul_rn(we / wv, P.cb));
        }
        const float2 a2 = __fmul2_rn(make_float2(lgu, q), make_float2(-2.0f, 2.0f));
        const float2 rs = sqrt_pos2(a2);  // (r, sd) = (sqrt(-2 ln u1), sqrt(2 q))
        const float r = rs.x, sd = rs.y;
        const float2 z = __fmul2_rn(make_float2(r, r), make_float2(cs, sn));
        // (xn, en) = ((xi, eta) + b) + sd z, the noise term fused
        const float2 n = __ffma2_rn(make_float2(sd, sd), z, __fadd2_rn(make_float2(xi, eta), b));
        if (!Mode<FL>::periodic(P)) {
            const float2 o = __ffma2_rn(n, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));  // 1 - xn, 1 - en
            // outside the square: v < 0 or 1 - v < 0 for v = xn or en, i.e. v (1 - v) < 0 (the two
            // cannot both be negative, and no product of these magnitudes rounds to zero)
            const float2 pr = __fmul2_rn(n, o);
            bool exited = fminf(pr.x, pr.y) < 0.0f;
            int s = -1;
            // The bridge test runs on every lane, without a branch: a lane that already left by
            // the endpoint test computes it too (its probabilities may be inf or NaN there) and
            // ignores the result.
            if (Mode<FL>::bridge(P)) {
                const float sc = __fdividef(-1.4426950408889634f, q);
                const float2 oi = __ffma2_rn(make_float2(xi, eta), make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
                const float2 a02 = __fmul2_rn(__fmul2_rn(make_float2(xi, eta), n), make_float2(sc, sc));
                const float2 a13 = __fmul2_rn(__fmul2_rn(oi, o), make_float2(sc, sc));
                float p0, p1, p2, p3;
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p0) : "f"(a02.x));
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p2) : "f"(a02.y));
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p1) : "f"(a13.x));
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p3) : "f"(a13.y));
                const float2 s01 = __ffma2_rn(make_float2(p0, p1), make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
                const float2 s23 = __ffma2_rn(make_float2(p2, p3), make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
                float surv = s01.x * s01.y;
                surv *= s23.x;
                surv *= s23.y;
                const bool bexit = !exited && ub > surv;
                float pm = p0;  // the side of the largest crossing probability
                int sb = 0;
                if (p1 > pm) { pm = p1; sb = 1; }
                if (p2 > pm) { pm = p2; sb = 2; }
                if (p3 > pm) { pm = p3; sb = 3; }
                s = bexit ? sb : -1;
                exited = exited || bexit;
            }
            if (exited) {
                vx = n.x;
                vy = n.y;
                side = s;
                return 1;
            }
        }
        xi = n.x;
        eta = n.y;
        return k + 1 == P.K ? 2 : 0;
    } else {
    const T u1 = uniform_open(w.x, T()), u2 = uniform_open(w.y, T()), ub = uniform_open(w.z, T());
    const T lgu = dlog(u1);
    T sn, cs;
    sincos(Consts<T>::two_pi * u2, &sn, &cs);
    T q, bx, by;  // q = D ds, (bx, by) = drift * ds
    if (!Mode<FL>::form1(P)) {
        q = wv * P.cb;
        bx = mul_rn(wx, P.cb);
        by = mul_rn(we, P.cb);
    } else {
        q = P.cb;
        bx = mul_rn(wx / wv, P.cb);
        by = mul_rn(we / wv, P.cb);
    }
    // Eq. 7: increment sqrt(2 q) z with the Box-Muller normals z = sqrt(-2 ln u1) (cos, sin)(2 pi u2),
    // operation for operation as the oracle: (xi + bx) + sd (r cos), each rounded
    const T r = dsqrt((T)-2 * lgu);
    const T sd = dsqrt(2 * q);
    const T xn = add_rn(add_rn(xi, bx), mul_rn(sd, mul_rn(r, cs)));
    const T en = add_rn(add_rn(eta, by), mul_rn(sd, mul_rn(r, sn)));

    if (!Mode<FL>::periodic(P)) {
        // outside the unit square: the largest violation is positive, i.e. the smallest of the
        // distances xn, 1 - xn, en, 1 - en is negative (1 - v is exactly -(v - 1) in floating
        // point, so the two forms decide alike); the distances serve the bridge test as well.
        // The side (ties keep the lower index) is found only for the paths that exit this way,
        // in the exit block.
        const T oxn = 1 - xn, oen = 1 - en;
        bool exited = dmin(dmin(xn, oxn), dmin(en, oen)) < 0;
        int s = -1;
        if (!exited && Mode<FL>::bridge(P)) {
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
        s2x = fma(dx, dx, s2x);
        s1y += dy;
        s2y = fma(dy, dy, s2y);
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
        // the square's compensated add: y = d^2 - c as one explicit fused operation
        const float2 y = __ffma2_rn(d, d, neg(c2));
        const float2 t = __fadd2_rn(s2, y);
        c2 = __fadd2_rn(__fadd2_rn(t, neg(s2)), neg(y));
        s2 = t;
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
        a = fma(-nn, ex, S1x);
        b = fma(nn * ex, ex, fma(-2.0 * ex, S1x, S2x));
        c = fma(-nn, ey, S1y);
        d = fma(nn * ey, ey, fma(-2.0 * ey, S1y, S2y));
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

template <typename T, int ACC, bool DEBUG, bool RK, int FL>
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
            const T vx = fma(R.Lx, fx, ix), vy = fma(R.Ly, fy, iy);
            acc.add(vx, vy);
            if (DEBUG) {
                const int64_t qd = checked((int64_t)q_path[pos] - P.dbg_p0, P.dbg_n);  // debug only
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
                const int64_t qd = checked((int64_t)Q.e_path[pos] - P.dbg_p0, P.dbg_n);  // debug only
                P.dbg_val[2 * qd] = (double)vx;
                P.dbg_val[2 * qd + 1] = (double)vy;
                P.dbg_steps[qd] = Q.e_k[pos];
                P.dbg_side[qd] = (int8_t)side;
            }
        }
        qe -= count;
        __syncwarp();
    };
    // Every lane runs a substep each iteration: a lane past the task's last path (live false)
    // runs a stale path whose results are masked, which keeps the loop free of a per-substep
    // vote and divergent branch.  Such a lane stays at its node or inside the domain (an exit
    // leaves its position unchanged), so its gathers stay in bounds.
    for (;;) {
        T vx, vy;
        int side = 0;
        int st = path_substep<T, RK, FL>(R, (uint32_t)m, path, k, xi, eta, vx, vy, side, ph);
        ++k;
        st = live ? st : 0;
        if (st != 0) {
            steps += (uint32_t)k;
            paths += 1;
        }
        const unsigned dm = __ballot_sync(kFull, st != 0);
        if (dm) {  // some lane's path ended: queue survivors and exits, hand out the next path indices
            const unsigned sm = __ballot_sync(kFull, st == 2);
            const int before = __popc(dm & lt);  // ended lanes below this one
            const int sbefore = __popc(sm & lt);  // of them, survivors
            if (st == 2) {
                const int pos = checked(qn + sbefore, 64);
                q_xi[pos] = xi;
                q_eta[pos] = eta;
                if (DEBUG) q_path[pos] = path;
            } else if (st == 1) {
                const int pos = checked(qe + before - sbefore, 64);
                Q.e_xn[pos] = vx;
                Q.e_en[pos] = vy;
                Q.e_side[pos] = side;
                if (DEBUG) {
                    Q.e_k[pos] = k;
                    Q.e_path[pos] = path;
                }
            }
            if (st != 0) {
                path = next + (uint32_t)before;
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
            const int ns = __popc(sm), nd = __popc(dm);
            qn += ns;
            qe += nd - ns;
            next += (uint32_t)nd;
            if ((qn | qe) >= 32) {  // both below 64
                if (qn >= 32) drain(32);
                if (qe >= 32) drain_exits(32);
            }
            if (!__any_sync(kFull, live)) break;
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
// FL: the problem switches compiled in (Mode; single-problem launches), or -1.
template <typename T, int ACC, bool DEBUG, bool BATCH, int TPB = kMcThreads, int FL = -1>
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
            run_task<T, ACC, DEBUG, false, FL>(P, R, g - R.node_offset, g, task, pb, pe, Q);
        } else {
            run_task<T, ACC, DEBUG, true, FL>(P, P.prob, g, g, task, pb, pe, Q);
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
                               int64_t* steps, int64_t* paths_run, int64_t* next_total, const int32_t* role,
                               int lo, int hi)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    acc[4 * m] = acc[4 * m + 1] = acc[4 * m + 2] = acc[4 * m + 3] = 0.0;
    n_done[m] = 0;
    steps[m] = 0;
    paths_run[m] = 0;
    const bool skipped = (role && role[m] >= 0) || m < lo || m >= hi;  // interpolated, or another range's
    next_total[m] = skipped ? 0 : (n0 < max_paths ? n0 : max_paths);
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

// The FP32 Box-Muller pieces of the path kernel on given Philox words: for each word w,
// u = uniform_open(w), ln u (log_unit), sqrt(-2 ln u) (sqrt_pos2), sin 2 pi u and cos 2 pi u.
__global__ void unit_math_kernel(const uint32_t* w, int64_t n, float* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float u = uniform_open(w[i], 0.0f);
    const float l = log_unit(u);
    const float r = sqrt_pos2(make_float2(-2.0f * l, u)).x;
    float sn, cs;
    sincos_2pi(u, &sn, &cs);
    float* o = out + 5 * i;
    o[0] = u;
    o[1] = l;
    o[2] = r;
    o[3] = sn;
    o[4] = cs;
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

// The path kernels gather the packed grids through L1.  Each kernel asks, once per device, for
// the smallest shared-memory carve-out that holds the per-warp queues of the blocks its registers
// let reside on an SM, so that the rest of the SM's unified L1 / shared memory serves as cache
// (left to itself the driver may pick a larger carve-out).
void prefer_l1(const void* fn, int tpb)
{
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!done.insert({fn, dev}).second) return;
    }
    cudaFuncAttributes fa{};
    int reserved = 0, max_smem = 0, max_threads = 0, regs_per_sm = 0;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        max_smem <= 0 || fa.numRegs <= 0) {
        cudaGetLastError();
        return;
    }
    int blocks = regs_per_sm / (fa.numRegs * tpb);
    blocks = std::max(1, std::min(blocks, max_threads / tpb));
    const long need = (long)blocks * ((long)fa.sharedSizeBytes + reserved);
    const int pct = (int)std::min(100L, (100 * need + max_smem - 1) / max_smem);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
        cudaGetLastError();  // a hint: the launch goes ahead with the driver's choice
}

template <typename T, int ACC, bool DEBUG, bool BATCH, int TPB, int FL>
void prefer_l1_for()
{
    prefer_l1(reinterpret_cast<const void*>(&mc_kernel<T, ACC, DEBUG, BATCH, TPB, FL>), TPB);
}

template <typename T, int TPB, int FL>
void launch_batch_mc_fl(const McParams<T>& P, bool kahan, int grid, cudaStream_t s)
{
    if (kahan) {
        prefer_l1_for<T, kAccKahan32, false, true, TPB, FL>();
        mc_kernel<T, kAccKahan32, false, true, TPB, FL><<<grid, TPB, 0, s>>>(P);
    } else {
        prefer_l1_for<T, kAcc64, false, true, TPB, FL>();
        mc_kernel<T, kAcc64, false, true, TPB, FL><<<grid, TPB, 0, s>>>(P);
    }
}

// A batch whose problems all share the Dirichlet / bridge-test / generator-form-0 switches
// (mode kModeDirichletBridge) runs the FP32 instantiation with them compiled in.
template <typename T, int TPB>
void launch_batch_mc_kernel(const McParams<T>& P, bool kahan, int grid, cudaStream_t s, int mode)
{
    if constexpr (sizeof(T) == 4) {
        if (mode == kModeDirichletBridge) {
            launch_batch_mc_fl<T, TPB, kModeDirichletBridge>(P, kahan, grid, s);
            return;
        }
    }
    launch_batch_mc_fl<T, TPB, -1>(P, kahan, grid, s);
}

// Single-problem FP32 launches of the common switch settings run a kernel with them compiled in
// (the same arithmetic without the per-substep branches); the rest the general kernel.
template <typename T, int ACC>
void launch_single_mc(const McParams<T>& P, int grid, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        const int mode = (P.prob.periodic ? 1 : 0) | (P.prob.form ? 2 : 0) | (P.prob.bb ? 4 : 0);
        if (mode == kModeDirichletBridge) {
            prefer_l1_for<T, ACC, false, false, kMcThreads, kModeDirichletBridge>();
            mc_kernel<T, ACC, false, false, kMcThreads, kModeDirichletBridge><<<grid, kMcThreads, 0, s>>>(P);
            return;
        }
        if (mode == kModeDirichletBridgeForm1) {
            prefer_l1_for<T, ACC, false, false, kMcThreads, kModeDirichletBridgeForm1>();
            mc_kernel<T, ACC, false, false, kMcThreads, kModeDirichletBridgeForm1><<<grid, kMcThreads, 0, s>>>(P);
            return;
        }
    }
    prefer_l1_for<T, ACC, false, false, kMcThreads, -1>();
    mc_kernel<T, ACC, false, false><<<grid, kMcThreads, 0, s>>>(P);
}

template <typename T>
cudaError_t launch_mc(const McParams<T>& P, int acc_mode, bool debug, bool batch, int grid, cudaStream_t s,
                      int tpb, int batch_mode)
{
    const bool kahan = acc_mode == kAccKahan32;
    if (batch) {
        if (tpb == 128) launch_batch_mc_kernel<T, 128>(P, kahan, grid, s, batch_mode);
        else if (tpb == 512) launch_batch_mc_kernel<T, 512>(P, kahan, grid, s, batch_mode);
        else launch_batch_mc_kernel<T, kMcThreads>(P, kahan, grid, s, batch_mode);
    } else if (debug) {
        if (kahan) {
            prefer_l1_for<T, kAccKahan32, true, false, kMcThreads, -1>();
            mc_kernel<T, kAccKahan32, true, false><<<grid, kMcThreads, 0, s>>>(P);
        } else {
            prefer_l1_for<T, kAcc64, true, false, kMcThreads, -1>();
            mc_kernel<T, kAcc64, true, false><<<grid, kMcThreads, 0, s>>>(P);
        }
    } else {
        if (kahan) launch_single_mc<T, kAccKahan32>(P, grid, s);
        else launch_single_mc<T, kAcc64>(P, grid, s);
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

template cudaError_t launch_mc<float>(const McParams<float>&, int, bool, bool, int, cudaStream_t, int, int);
template cudaError_t launch_mc<double>(const McParams<double>&, int, bool, bool, int, cudaStream_t, int, int);
template int mc_max_blocks_per_sm<float>(int, bool, bool, int);
template int mc_max_blocks_per_sm<double>(int, bool, bool, int);

cudaError_t launch_mc_init(int M, int64_t n0, int64_t max_paths, double* acc, int64_t* n_done,
                           int64_t* steps, int64_t* paths_run, int64_t* next_total, cudaStream_t s,
                           const int32_t* role, int lo, int hi)
{
    mc_init_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, n0, max_paths, acc, n_done, steps, paths_run,
                                                   next_total, role, lo, hi < 0 ? M : hi);
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

cudaError_t launch_unit_math(const uint32_t* w, int64_t n, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    unit_math_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, n, out);
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
