/*
 * Path simulator body of the SDD oracle (TEST INFRASTRUCTURE; see sdd_oracle.c).
 * Included twice by sdd_oracle.c with REAL = double / float and SFX = f64 / f32.
 *
 * Notation follows the paper: the computational coordinates are xi = (xi, eta) in the unit
 * square, the monitor (mesh density) is omega, the SDE of Eq. (5b) is stepped by the
 * Euler-Maruyama scheme of Eq. (7) with K substeps of length ds = dt / K, and a path that
 * started at an interface node contributes either the boundary value at its exit point
 * (second term of Eq. 5a) or the previous mesh interpolated at its final position
 * (first term of Eq. 5a, and Eq. 6 on periodic domains).
 *
 * Generator forms (both relax the linearised mesh PDE with time constant tau):
 *   form 0:  tau x_t = div(omega grad x)                   drift grad(omega)/tau,          D = omega/tau
 *   form 1:  tau x_t = grad(omega)/omega . grad x + lap x  drift grad(omega)/(omega tau),  D = 1/tau
 * (form 1 with tau = 1 is the paper's Eq. 4 and Eq. 5b).  D is the diffusion coefficient:
 * the noise amplitude of Eq. (7) is sqrt(2 D ds).
 */
#define NAME(x) CAT2(x, SFX)

#if REAL_IS_FLOAT
#define R_LOG logf
#define R_SQRT sqrtf
#define R_COS cosf
#define R_SIN sinf
#define R_EXP expf
#define R_FLOOR floorf
#define R_FABS fabsf
#define R_TWO_PI 6.28318530717958647692f
#else
#define R_LOG log
#define R_SQRT sqrt
#define R_COS cos
#define R_SIN sin
#define R_EXP exp
#define R_FLOOR floor
#define R_FABS fabs
#define R_TWO_PI 6.28318530717958647692
#endif

typedef struct {
    int32_t nx, ny;      /* nodes per direction of the computational grid (>= 3)               */
    int32_t periodic;    /* 0: Dirichlet, boundary mesh x = (Lx xi, Ly eta); 1: doubly periodic */
    int32_t form;        /* 0 or 1, see above                                                    */
    int32_t K;           /* substeps per time step                                               */
    int32_t bicubic;     /* 1: Keys bicubic for the previous mesh, 0: bilinear                  */
    int32_t bb_test;     /* 1: Brownian-bridge crossing test between substeps (Dirichlet only)  */
    int32_t tstep;       /* time-step index n (fourth Philox counter word)                      */
    uint32_t key0, key1; /* Philox key (the 64-bit seed, low word first)                        */
    double Lx, Ly;       /* physical rectangle [0, Lx] x [0, Ly]                                 */
    double tau, dt;      /* relaxation time and mesh time step                                   */
    const REAL* w;       /* omega at the nodes, row-major [j * nx + i]                           */
    const REAL* w_xi;    /* d omega / d xi at the nodes (finite differences, Sec. 3.4)           */
    const REAL* w_eta;   /* d omega / d eta at the nodes                                         */
    const REAL* X;       /* previous mesh displacement x - Lx xi at the nodes                    */
    const REAL* Y;       /* previous mesh displacement y - Ly eta at the nodes                   */
    const REAL* bnd;     /* moving boundary (NULL: the identity): tangential coordinate of the
                            new boundary mesh, x on eta = 0 (nx values) and eta = 1 (nx), then y
                            on xi = 0 (ny) and xi = 1 (ny)                                      */
} NAME(oracle_problem);

/* Linear interpolation of the n values b (nodes s = k / (n - 1)) at s in [0, 1]. */
static REAL NAME(side_lerp)(const REAL* b, int n, REAL s)
{
    REAL u = s * (REAL)(n - 1);
    REAL fl = R_FLOOR(u);
    long c = (long)fl;
    if (c < 0) c = 0;
    if (c > n - 2) c = n - 2;
    REAL f = u - (REAL)c;
    return ((REAL)1 - f) * b[c] + f * b[c + 1];
}

/* Uniform deviate in (0, 1) from one 32-bit Philox word, formed without rounding:
 * FP64: (w + 1/2) 2^-32;  FP32: (floor(w / 2^9) + 1/2) 2^-23 (24 significant bits). */
static REAL NAME(uniform)(uint32_t w)
{
#if REAL_IS_FLOAT
    return ((float)(w >> 9) + 0.5f) * 0x1p-23f;
#else
    return ((double)w + 0.5) * 0x1p-32;
#endif
}

/* Box-Muller: two independent N(0,1) deviates from two uniforms (the N(0,1) of Eq. 7). */
static void NAME(box_muller)(REAL u1, REAL u2, REAL* z1, REAL* z2)
{
    REAL r = R_SQRT((REAL)-2 * R_LOG(u1));
    REAL angle = R_TWO_PI * u2;
    *z1 = r * R_COS(angle);
    *z2 = r * R_SIN(angle);
}

/* Cell containing coordinate s of an n-node grid on [0, 1] and the offset inside it.
 * Dirichlet: cells 0 .. n-2 (s = 1 falls in the last cell with offset 1).
 * Periodic: the grid repeats with period 1 (n - 1 distinct nodes, node n-1 equals node 0). */
static void NAME(locate)(int n, int periodic, REAL s, int* cell, REAL* frac)
{
    REAL u = s * (REAL)(n - 1);
    REAL fl = R_FLOOR(u);
    long c = (long)fl;
    if (periodic) {
        long m = n - 1;
        c %= m;
        if (c < 0) c += m;
        *frac = u - fl;
    } else {
        if (c < 0) c = 0;
        if (c > n - 2) c = n - 2;
        *frac = u - (REAL)c;
    }
    *cell = (int)c;
}

/* Bilinear interpolation of the nodal field f at (xi, eta) (Sec. 3.4). */
static REAL NAME(bilinear)(int nx, int ny, int periodic, const REAL* f, REAL xi, REAL eta)
{
    int i, j;
    REAL fx, fy;
    NAME(locate)(nx, periodic, xi, &i, &fx);
    NAME(locate)(ny, periodic, eta, &j, &fy);
    REAL f00 = f[j * nx + i], f10 = f[j * nx + i + 1];
    REAL f01 = f[(j + 1) * nx + i], f11 = f[(j + 1) * nx + i + 1];
    return (1 - fx) * (1 - fy) * f00 + fx * (1 - fy) * f10 + (1 - fx) * fy * f01 + fx * fy * f11;
}

/* Keys (1981) cubic-convolution kernel with a = -1/2. */
static REAL NAME(keys_kernel)(REAL s)
{
    const REAL a = (REAL)-0.5;
    s = R_FABS(s);
    if (s <= 1) return (a + 2) * s * s * s - (a + 3) * s * s + 1;
    if (s < 2) return a * s * s * s - 5 * a * s * s + 8 * a * s - 4 * a;
    return 0;
}

/* 1-D cubic convolution through samples at offsets -1, 0, 1, 2 for a point at offset t. */
static REAL NAME(keys_1d)(const REAL g[4], REAL t)
{
    return g[0] * NAME(keys_kernel)(1 + t) + g[1] * NAME(keys_kernel)(t) +
           g[2] * NAME(keys_kernel)(1 - t) + g[3] * NAME(keys_kernel)(2 - t);
}

/* Value of row j of f at columns cell-1 .. cell+2, then interpolated at offset t.
 * Dirichlet: a column outside the grid is Keys' boundary extrapolation
 * f(-1) = 3 f(0) - 3 f(1) + f(2) (and its mirror at the right end).
 * Periodic: columns wrap with period nx - 1. */
static REAL NAME(keys_row)(int nx, int periodic, const REAL* row, int cell, REAL t)
{
    REAL g[4];
    if (periodic) {
        int m = nx - 1;
        for (int a = 0; a < 4; ++a) {
            int c = ((cell - 1 + a) % m + m) % m;
            g[a] = row[c];
        }
    } else {
        for (int a = 0; a < 4; ++a) {
            int c = cell - 1 + a;
            if (c < 0)
                g[a] = 3 * row[0] - 3 * row[1] + row[2];
            else if (c > nx - 1)
                g[a] = 3 * row[nx - 1] - 3 * row[nx - 2] + row[nx - 3];
            else
                g[a] = row[c];
        }
    }
    return NAME(keys_1d)(g, t);
}

/* Tensor-product cubic convolution of the nodal field f at (xi, eta) (the "bi-cubic"
 * interpolation of the previous mesh in Sec. 3.4).  Rows are interpolated along xi first;
 * a row outside a Dirichlet grid is Keys' extrapolation of the interpolated rows. */
static REAL NAME(bicubic)(int nx, int ny, int periodic, const REAL* f, REAL xi, REAL eta)
{
    int i, j;
    REAL tx, ty;
    NAME(locate)(nx, periodic, xi, &i, &tx);
    NAME(locate)(ny, periodic, eta, &j, &ty);
    REAL g[4];
    if (periodic) {
        int m = ny - 1;
        for (int b = 0; b < 4; ++b) {
            int r = ((j - 1 + b) % m + m) % m;
            g[b] = NAME(keys_row)(nx, 1, f + (long)r * nx, i, tx);
        }
    } else {
        for (int b = 0; b < 4; ++b) {
            int r = j - 1 + b;
            if (r >= 0 && r <= ny - 1) g[b] = NAME(keys_row)(nx, 0, f + (long)r * nx, i, tx);
        }
        if (j - 1 < 0) g[0] = 3 * g[1] - 3 * g[2] + g[3];   /* rows 0, 1, 2 */
        if (j + 2 > ny - 1) g[3] = 3 * g[2] - 3 * g[1] + g[0]; /* rows ny-1, ny-2, ny-3 */
    }
    return NAME(keys_1d)(g, ty);
}

static REAL NAME(clamp01)(REAL v) { return v < 0 ? (REAL)0 : (v > 1 ? (REAL)1 : v); }

/* Index of the largest of four values; ties go to the lowest index. */
static int NAME(argmax4)(const REAL v[4])
{
    int s = 0;
    for (int t = 1; t < 4; ++t)
        if (v[t] > v[s]) s = t;
    return s;
}

/* Gap between the largest and the second largest of four values. */
static double NAME(gap4)(const REAL v[4], int s)
{
    double second = -INFINITY;
    for (int t = 0; t < 4; ++t)
        if (t != s && (double)v[t] > second) second = (double)v[t];
    return (double)v[s] - second;
}

/*
 * One path started at node (i0, j0) with node id m and path index p.
 *
 * Substep k draws Philox4x32-10 with counter (k, p, m, n) and key (key0, key1) -> words
 * (w0, w1, w2, w3); w0, w1 give the two normals of Eq. (7) by Box-Muller and w2 the uniform
 * of the Brownian-bridge test (w3 is unused).
 *
 * Boundary test (Dirichlet), for the proposed point phi' = phi + b ds + sqrt(2 D ds) z:
 *   - if phi' lies outside the unit square, the path exits through the side it violates
 *     most (ties: xi=0, xi=1, eta=0, eta=1); the exit point keeps the other coordinate of
 *     phi', clamped to [0, 1];
 *   - otherwise, with distances d0_s of phi and d1_s of phi' to each side s, the bridge
 *     crosses side s with probability exp(-d0_s d1_s / (D ds)); the path exits if the
 *     uniform exceeds prod_s (1 - p_s), through the side of largest p_s, at the point on
 *     that side that keeps phi''s other coordinate.
 * The exit value is the boundary mesh at the exit point: (Lx xi_e, Ly eta_e), or with a
 * moving boundary (Sec. 2) the new boundary mesh linearly interpolated along the exit side.  A path that
 * completes K substeps takes the previous mesh at its final point: (Lx xi_K + X(phi_K),
 * Ly eta_K + Y(phi_K)) with X, Y interpolated (periodic: indices wrap, the linear part
 * carries the period offset).
 *
 * Outputs: value (vx, vy); steps = substeps taken; side 0..3 = exit side, 4 = completed;
 * margin = the smallest distance of any boundary decision from its threshold (used by the
 * tests to tell robust decisions from near ties).
 */
void NAME(oracle_path)(const NAME(oracle_problem)* P, uint32_t m, int i0, int j0, uint32_t p,
                       double* vx, double* vy, int32_t* steps, int32_t* side, double* margin)
{
    const int nx = P->nx, ny = P->ny, per = P->periodic;
    REAL xi = (REAL)i0 / (REAL)(nx - 1);
    REAL eta = (REAL)j0 / (REAL)(ny - 1);
    const REAL ds = (REAL)P->dt / (REAL)P->K;
    const REAL cb = ds / (REAL)P->tau; /* ds / tau */
    const REAL Lx = (REAL)P->Lx, Ly = (REAL)P->Ly;
    double mg = INFINITY;

    for (int k = 0; k < P->K; ++k) {
        uint32_t ctr[4] = {(uint32_t)k, p, m, (uint32_t)P->tstep};
        uint32_t key[2] = {P->key0, P->key1};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        REAL z1, z2;
        NAME(box_muller)(NAME(uniform)(w[0]), NAME(uniform)(w[1]), &z1, &z2);
        REAL ub = NAME(uniform)(w[2]);

        /* Coefficients of Eq. (7) at phi^k from the bilinearly interpolated monitor. */
        REAL wv = NAME(bilinear)(nx, ny, per, P->w, xi, eta);
        REAL wx = NAME(bilinear)(nx, ny, per, P->w_xi, xi, eta);
        REAL we = NAME(bilinear)(nx, ny, per, P->w_eta, xi, eta);
        REAL q, bx, by; /* q = D ds; (bx, by) = drift * ds */
        if (P->form == 0) {
            q = wv * cb;
            bx = wx * cb;
            by = we * cb;
        } else {
            q = cb;
            bx = wx / wv * cb;
            by = we / wv * cb;
        }
        REAL sd = R_SQRT(2 * q);
        REAL xn = xi + bx + sd * z1;
        REAL en = eta + by + sd * z2;

        if (!per) {
            REAL viol[4] = {-xn, xn - 1, -en, en - 1};
            int s = NAME(argmax4)(viol);
            double dist = R_FABS(viol[s]);
            if (dist < mg) mg = dist;
            int exited = 0;
            if (viol[s] > 0) {
                exited = 1;
                double g = NAME(gap4)(viol, s);
                if (g < mg) mg = g;
            } else if (P->bb_test) {
                REAL d0[4] = {xi, 1 - xi, eta, 1 - eta};
                REAL d1[4] = {xn, 1 - xn, en, 1 - en};
                REAL pr[4];
                REAL surv = 1;
                for (int t = 0; t < 4; ++t) {
                    pr[t] = R_EXP(-(d0[t] * d1[t]) / q);
                    surv *= (1 - pr[t]);
                }
                double gm = R_FABS(ub - surv);
                if (gm < mg) mg = gm;
                if (ub > surv) {
                    exited = 1;
                    s = NAME(argmax4)(pr);
                    double g = NAME(gap4)(pr, s);
                    if (g < mg) mg = g;
                }
            }
            if (exited) {
                REAL xe = NAME(clamp01)(xn), ee = NAME(clamp01)(en);
                if (s == 0) xe = 0;
                if (s == 1) xe = 1;
                if (s == 2) ee = 0;
                if (s == 3) ee = 1;
                if (P->bnd) {   /* the new boundary mesh along the exit side */
                    const REAL* b = P->bnd;
                    REAL bx, by;
                    if (s == 0) { bx = 0; by = NAME(side_lerp)(b + 2 * nx, ny, ee); }
                    else if (s == 1) { bx = Lx; by = NAME(side_lerp)(b + 2 * nx + ny, ny, ee); }
                    else if (s == 2) { bx = NAME(side_lerp)(b, nx, xe); by = 0; }
                    else { bx = NAME(side_lerp)(b + nx, nx, xe); by = Ly; }
                    *vx = (double)bx;
                    *vy = (double)by;
                } else {
                    *vx = (double)(Lx * xe);
                    *vy = (double)(Ly * ee);
                }
                *steps = k + 1;
                *side = s;
                *margin = mg;
                return;
            }
        }
        xi = xn;
        eta = en;
    }

    REAL ix, iy;
    if (P->bicubic) {
        ix = NAME(bicubic)(nx, ny, per, P->X, xi, eta);
        iy = NAME(bicubic)(nx, ny, per, P->Y, xi, eta);
    } else {
        ix = NAME(bilinear)(nx, ny, per, P->X, xi, eta);
        iy = NAME(bilinear)(nx, ny, per, P->Y, xi, eta);
    }
    *vx = (double)(Lx * xi + ix);
    *vy = (double)(Ly * eta + iy);
    *steps = P->K;
    *side = 4;
    *margin = mg;
}

/* Per-path records for paths p_begin .. p_begin + n - 1 of node m (parity hook). */
void NAME(oracle_paths)(const NAME(oracle_problem)* P, uint32_t m, int i0, int j0, int64_t p_begin,
                        int64_t n, double* val_xy, int32_t* steps, int8_t* side, double* margin)
{
    for (int64_t q = 0; q < n; ++q) {
        int32_t st, sd;
        double mg;
        NAME(oracle_path)(P, m, i0, j0, (uint32_t)(p_begin + q), &val_xy[2 * q], &val_xy[2 * q + 1],
                          &st, &sd, &mg);
        steps[q] = st;
        side[q] = (int8_t)sd;
        margin[q] = mg;
    }
}

/*
 * Estimator sums of Sec. 3.4 for M nodes: node r (id node_id[r], grid position ij[2r],
 * ij[2r+1]) runs paths p_begin[r] .. p_begin[r] + n_paths[r] - 1 and accumulates, in path
 * order and in FP64, the shifted sums
 *   sums[4r+0] = sum (vx - shift_x),  sums[4r+1] = sum (vx - shift_x)^2,
 *   sums[4r+2] = sum (vy - shift_y),  sums[4r+3] = sum (vy - shift_y)^2,
 * and steps[r] = total substeps taken.  Nodes are independent (OpenMP over nodes).
 */
void NAME(oracle_interface_sums)(const NAME(oracle_problem)* P, int64_t M, const int32_t* node_id,
                                 const int32_t* ij, const int64_t* p_begin, const int64_t* n_paths,
                                 const double* shift_xy, double* sums, int64_t* steps)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < M; ++r) {
        double s1x = 0, s2x = 0, s1y = 0, s2y = 0;
        int64_t st_total = 0;
        for (int64_t q = 0; q < n_paths[r]; ++q) {
            double vx, vy, mg;
            int32_t st, sd;
            NAME(oracle_path)(P, (uint32_t)node_id[r], ij[2 * r], ij[2 * r + 1],
                              (uint32_t)(p_begin[r] + q), &vx, &vy, &st, &sd, &mg);
            double dx = vx - shift_xy[2 * r], dy = vy - shift_xy[2 * r + 1];
            s1x += dx;
            s2x += dx * dx;
            s1y += dy;
            s2y += dy * dy;
            st_total += st;
        }
        sums[4 * r + 0] = s1x;
        sums[4 * r + 1] = s2x;
        sums[4 * r + 2] = s1y;
        sums[4 * r + 3] = s2y;
        steps[r] = st_total;
    }
}

/* Exposed pieces for the tests. */
void NAME(oracle_box_muller)(uint32_t w0, uint32_t w1, double* z1, double* z2)
{
    REAL a, b;
    NAME(box_muller)(NAME(uniform)(w0), NAME(uniform)(w1), &a, &b);
    *z1 = (double)a;
    *z2 = (double)b;
}

double NAME(oracle_uniform)(uint32_t w) { return (double)NAME(uniform)(w); }

void NAME(oracle_interp)(int nx, int ny, int periodic, int bicubic, const REAL* f, int64_t n,
                         const double* pts, double* out)
{
    for (int64_t q = 0; q < n; ++q) {
        REAL a = (REAL)pts[2 * q], b = (REAL)pts[2 * q + 1];
        out[q] = (double)(bicubic ? NAME(bicubic)(nx, ny, periodic, f, a, b)
                                  : NAME(bilinear)(nx, ny, periodic, f, a, b));
    }
}

#undef NAME
#undef R_LOG
#undef R_SQRT
#undef R_COS
#undef R_SIN
#undef R_EXP
#undef R_FLOOR
#undef R_FABS
#undef R_TWO_PI
