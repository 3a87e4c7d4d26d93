/*
 * Plain FP64 CPU oracle for the tracer-advection hot path of
 * Lalescu, Bramas, Rampp & Wilczek, "An Efficient Particle Tracking Algorithm
 * for Large-Scale Parallel Pseudo-Spectral Simulations of Turbulence"
 * (arXiv:2107.01104).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Everything is IEEE double precision (the paper computes in double, Sec. 4.2).
 * Compile with -ffp-contract=off so that no multiply-add is fused: the cell
 * split below must round exactly like the GPU side for bit-exact binning.
 *
 * Layout conventions (stated once, used everywhere):
 *   positions   pos[3][np]      SoA, axis-major, x1 first; unwrapped (any real value)
 *   field       f[C][N][N][N]   component-major, then x3 (slowest), x2, x1 (fastest),
 *                               matching the x3-slab convention of Sec. 3.2
 *   outputs     out[C][np]
 *
 * Parity notes (what pins each function) live in the test suite; every
 * function here has at least one pin other than itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_I 8
#define ORC_MAX_DEG 12

/* ------------------------------------------------------------------------ */
/* Position split: Sec. 2.2, interpolation steps 1-3.                        */
/*                                                                          */
/* The paper forms X~ = X mod 2pi, picks the grid cell c of X~ and uses the */
/* offset x_bar = X~ - c*delta, normalised as x_bar/delta.  Rounding is not */
/* specified there; this oracle fixes it as                                 */
/*     g  = X * (N/L)           one IEEE multiply by fl(N/L)                */
/*     c0 = floor(g)            exact                                       */
/*     t  = g - c0              one IEEE subtraction, t in [0,1]            */
/*     c  = c0 mod N            Euclidean, in [0,N)                         */
/* which is the same number up to rounding, and is what the GPU reproduces  */
/* bit for bit.  The cell is the one whose lower corner is at or below X~:  */
/* the node range 1-I/2..I/2 of Eq. (triple_sum) is centred on [0,1).       */
/* ------------------------------------------------------------------------ */
static int split_one(double X, int N, double inv_delta, int32_t* c, double* t)
{
    if (!isfinite(X)) return -1;
    double g = X * inv_delta;
    double c0 = floor(g);
    *t = g - c0;
    double r = fmod(c0, (double)N);
    if (r < 0) r += (double)N;
    *c = (int32_t)r;
    return 0;
}

double orc_inv_delta(int N, double L) { return (double)N / L; }

int orc_split(int64_t np, const double* pos, int N, double L, int32_t* cell, double* frac)
{
    double inv_delta = orc_inv_delta(N, L);
    int bad = 0;
    for (int64_t p = 0; p < np; ++p)
        for (int a = 0; a < 3; ++a)
            if (split_one(pos[a * np + p], N, inv_delta, &cell[a * np + p], &frac[a * np + p])) bad = 1;
    return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* Small dense linear solve (Gaussian elimination, partial pivoting).        */
/* Used only to build the spline polynomials procedurally.                  */
/* ------------------------------------------------------------------------ */
static void solve_dense(int n, double* A /* n*n row-major, destroyed */, double* b /* n, overwritten by x */)
{
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (piv != col) {
            for (int k = 0; k < n; ++k) { double tmp = A[col * n + k]; A[col * n + k] = A[piv * n + k]; A[piv * n + k] = tmp; }
            double tmp = b[col]; b[col] = b[piv]; b[piv] = tmp;
        }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r * n + col] / A[col * n + col];
            for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
}

static double factorial(int q) { double f = 1; for (int i = 2; i <= q; ++i) f *= i; return f; }

/* ------------------------------------------------------------------------ */
/* Lagrange weights (Sec. 2.2: "simple Lagrange interpolation schemes").     */
/* Nodes j in S = {1-I/2, ..., I/2} relative to the cell; textbook product   */
/*     beta_i(t) = prod_{j in S, j != i} (t - j) / (i - j).                  */
/* beta[k] holds the weight of node i = k + 1 - I/2.                         */
/* ------------------------------------------------------------------------ */
static void lagrange_weights(int I, double t, double* beta, double* dbeta)
{
    int lo = 1 - I / 2;
    for (int a = 0; a < I; ++a) {
        int i = lo + a;
        double prod = 1.0;
        for (int b = 0; b < I; ++b) {
            int j = lo + b;
            if (j == i) continue;
            prod *= (t - j) / (double)(i - j);
        }
        beta[a] = prod;
        if (dbeta) {
            /* d/dt of the product: sum over the factor that is differentiated */
            double s = 0.0;
            for (int k = 0; k < I; ++k) {
                int kk = lo + k;
                if (kk == i) continue;
                double term = 1.0 / (double)(i - kk);
                for (int b = 0; b < I; ++b) {
                    int j = lo + b;
                    if (j == i || j == kk) continue;
                    term *= (t - j) / (double)(i - j);
                }
                s += term;
            }
            dbeta[a] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Spline weights, family of Sec. 2.2 [ref. lalescu2010jcp].                  */
/*                                                                          */
/* The cited construction is not reproduced in the paper; this oracle uses  */
/* the reading: I = 2n+2 nodes {-n..n+1}; on the cell [0,1] the interpolant */
/* is the polynomial of degree 2m+1 whose derivatives of order 0..m at      */
/* t = 0 and t = 1 equal those of the centred (2n+1)-point Lagrange          */
/* polynomial through nodes p-n..p+n (p = 0, 1).  Neighbouring cells share   */
/* node derivatives, so the interpolant is C^m.  Built procedurally:         */
/*   (a) node derivatives: solve the Vandermonde system of the centred       */
/*       stencil, derivative q = q! * (monomial coefficient q);             */
/*   (b) two-point Hermite problem: solve for the 2m+2 monomial coefficients;*/
/*   (c) evaluate at t.                                                      */
/* beta_i(t) is the interpolant of the unit vector e_i.                      */
/* ------------------------------------------------------------------------ */
static void node_derivatives(int n, int m, const double* y /* values on nodes -n..n+1 */, int p, double* D /* m+1 */)
{
    int K = 2 * n + 1;
    double A[ORC_MAX_DEG * ORC_MAX_DEG], b[ORC_MAX_DEG];
    for (int r = 0; r < K; ++r) {
        double x = (double)(r - n); /* node p-n+r, relative to p */
        double xp = 1.0;
        for (int s = 0; s < K; ++s) { A[r * K + s] = xp; xp *= x; }
        b[r] = y[(p - n + r) + n]; /* index into nodes -n..n+1 */
    }
    solve_dense(K, A, b);
    for (int q = 0; q <= m; ++q) D[q] = (q < K) ? factorial(q) * b[q] : 0.0;
}

static void spline_poly(int n, int m, const double* y, double* h /* 2m+2 monomial coefficients in t */)
{
    double D0[ORC_MAX_DEG], D1[ORC_MAX_DEG];
    node_derivatives(n, m, y, 0, D0);
    node_derivatives(n, m, y, 1, D1);
    int K = 2 * m + 2;
    double A[ORC_MAX_DEG * ORC_MAX_DEG];
    memset(A, 0, sizeof(A));
    for (int q = 0; q <= m; ++q) {
        /* P^(q)(0) = q! h_q */
        for (int s = 0; s < K; ++s) A[q * K + s] = (s == q) ? factorial(q) : 0.0;
        h[q] = D0[q];
        /* P^(q)(1) = sum_{s>=q} s!/(s-q)! h_s */
        for (int s = 0; s < K; ++s) A[(m + 1 + q) * K + s] = (s >= q) ? factorial(s) / factorial(s - q) : 0.0;
        h[m + 1 + q] = D1[q];
    }
    solve_dense(K, A, h);
}

static void spline_weights(int I, int m, double t, double* beta, double* dbeta)
{
    int n = I / 2 - 1;
    int K = 2 * m + 2;
    for (int a = 0; a < I; ++a) {
        double y[ORC_MAX_I];
        for (int b = 0; b < I; ++b) y[b] = (a == b) ? 1.0 : 0.0;
        double h[ORC_MAX_DEG];
        spline_poly(n, m, y, h);
        double v = 0.0, dv = 0.0, tp = 1.0;
        for (int s = 0; s < K; ++s) { v += h[s] * tp; tp *= t; }
        tp = 1.0;
        for (int s = 1; s < K; ++s) { dv += s * h[s] * tp; tp *= t; }
        beta[a] = v;
        if (dbeta) dbeta[a] = dv;
    }
}

/* family: 0 Lagrange, 1 spline.  Returns 0, or -1 for unsupported (I, m). */
int orc_check_kernel(int family, int I, int m)
{
    if (I != 4 && I != 6 && I != 8) return -1;
    if (family == 0) return 0;
    if (family != 1) return -1;
    int n = I / 2 - 1;
    if (m < 0 || m > n + 1) return -1;
    return 0;
}

int orc_weights(int family, int I, int m, double t, double* beta, double* dbeta)
{
    if (orc_check_kernel(family, I, m)) return -1;
    if (family == 0) lagrange_weights(I, t, beta, dbeta);
    else spline_weights(I, m, t, beta, dbeta);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Binning: Sec. 3.3.1 "Ordering the particles locally".                     */
/* The paper groups particles by x3 slice and stores offset[s] (start of     */
/* group s, with offset[Ps] = number of particles).  Here the groups are     */
/* blocks of B1 x B2 x B3 cells, x3-major (B = 1 gives one group per cell;   */
/* B1 = B2 = N gives the paper's slices).  The order inside a group is the   */
/* incoming order: a stable counting sort by block key.                      */
/*   key  = (c3/B3 * (N/B2) + c2/B2) * (N/B1) + c1/B1                        */
/*   perm[j]  = incoming index of the particle at sorted position j          */
/*   offsets[b] = first sorted position of group b; offsets[nblocks] = np    */
/* ------------------------------------------------------------------------ */
int orc_bin(int64_t np, const double* pos, int N, double L, int B1, int B2, int B3,
            int32_t* keys, int64_t* perm, int64_t* offsets)
{
    if (B1 <= 0 || B2 <= 0 || B3 <= 0 || N % B1 || N % B2 || N % B3) return -1;
    double inv_delta = orc_inv_delta(N, L);
    int64_t nb1 = N / B1, nb2 = N / B2, nb3 = N / B3;
    int64_t nblocks = nb1 * nb2 * nb3;
    int bad = 0;
    for (int64_t p = 0; p < np; ++p) {
        int32_t c[3]; double t;
        for (int a = 0; a < 3; ++a)
            if (split_one(pos[a * np + p], N, inv_delta, &c[a], &t)) { bad = 1; c[a] = 0; }
        keys[p] = (int32_t)(((int64_t)(c[2] / B3) * nb2 + c[1] / B2) * nb1 + c[0] / B1);
    }
    if (bad) return -4;
    /* stable counting sort: count, exclusive prefix, place in incoming order */
    memset(offsets, 0, (size_t)(nblocks + 1) * sizeof(int64_t));
    for (int64_t p = 0; p < np; ++p) offsets[keys[p] + 1] += 1;
    for (int64_t b = 0; b < nblocks; ++b) offsets[b + 1] += offsets[b];
    int64_t* next = (int64_t*)malloc((size_t)nblocks * sizeof(int64_t));
    if (!next) return -2;
    memcpy(next, offsets, (size_t)nblocks * sizeof(int64_t));
    for (int64_t p = 0; p < np; ++p) perm[next[keys[p]]++] = p;
    free(next);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Interpolation: Sec. 2.2, step 4, Eq. (triple_sum).                        */
/*   u(X) = sum_{i1,i2,i3 = 1-I/2}^{I/2} beta_i1(t1) beta_i2(t2) beta_i3(t3) */
/*          u(c + i)                                                        */
/* with periodic node indices (the domain is periodic, Sec. 2.1).  Written   */
/* as the direct quadruple loop: no separable reuse (the CUDA path uses the  */
/* separable order of Sec. 3.3, so agreement also checks that split).        */
/* deriv = 1 returns d u_k / d X_j (out[(k*3 + j)*np + p]): beta' on axis j, */
/* times N/L, the derivative of t with respect to X.                         */
/* ------------------------------------------------------------------------ */
struct orc_kernel { int family, I, m; };

static void interp_one(const struct orc_kernel* K, const double* f, int C, int N, double inv_delta,
                       const int32_t* c, const double* t, int deriv, double* res /* C or 3C */)
{
    int I = K->I;
    double w[3][ORC_MAX_I], dw[3][ORC_MAX_I];
    for (int a = 0; a < 3; ++a) orc_weights(K->family, I, K->m, t[a], w[a], dw[a]);
    int lo = 1 - I / 2;
    int64_t NN = N;
    int nout = deriv ? 3 * C : C;
    for (int r = 0; r < nout; ++r) res[r] = 0.0;
    for (int a3 = 0; a3 < I; ++a3) {
        int64_t x3 = ((c[2] + lo + a3) % N + N) % N;
        for (int a2 = 0; a2 < I; ++a2) {
            int64_t x2 = ((c[1] + lo + a2) % N + N) % N;
            for (int a1 = 0; a1 < I; ++a1) {
                int64_t x1 = ((c[0] + lo + a1) % N + N) % N;
                int64_t node = (x3 * NN + x2) * NN + x1;
                for (int k = 0; k < C; ++k) {
                    double v = f[(int64_t)k * NN * NN * NN + node];
                    if (!deriv) {
                        res[k] += w[0][a1] * w[1][a2] * w[2][a3] * v;
                    } else {
                        res[k * 3 + 0] += dw[0][a1] * w[1][a2] * w[2][a3] * v * inv_delta;
                        res[k * 3 + 1] += w[0][a1] * dw[1][a2] * w[2][a3] * v * inv_delta;
                        res[k * 3 + 2] += w[0][a1] * w[1][a2] * dw[2][a3] * v * inv_delta;
                    }
                }
            }
        }
    }
}

int orc_interp(int family, int I, int m, int N, double L, const double* field, int C,
               int64_t np, const double* pos, double* out, int deriv)
{
    struct orc_kernel K = { family, I, m };
    if (orc_check_kernel(family, I, m)) return -1;
    double inv_delta = orc_inv_delta(N, L);
    int bad = 0;
    int nout = deriv ? 3 * C : C;
    #pragma omp parallel for schedule(dynamic, 256) reduction(|:bad)
    for (int64_t p = 0; p < np; ++p) {
        int32_t c[3]; double t[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a) if (split_one(pos[a * np + p], N, inv_delta, &c[a], &t[a])) ok = 0;
        double res[3 * 16];
        if (!ok) { bad = 1; for (int r = 0; r < nout; ++r) out[r * np + p] = NAN; continue; }
        interp_one(&K, field, C, N, inv_delta, c, t, deriv, res);
        for (int r = 0; r < nout; ++r) out[r * np + p] = res[r];
    }
    return bad ? -4 : 0;
}

/* Interpolation from pre-gathered stencils (for fields too large to hold on */
/* the host): stencil[p][k][a3][a2][a1] holds u_k at node c + (a - I/2 + 1), */
/* frac[3][np] the offsets t.  Same triple sum as above.                     */
int orc_interp_stencil(int family, int I, int m, int C, int64_t np, const double* frac,
                       const double* stencil, double* out)
{
    if (orc_check_kernel(family, I, m)) return -1;
    int64_t I3 = (int64_t)I * I * I;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < np; ++p) {
        double w[3][ORC_MAX_I];
        for (int a = 0; a < 3; ++a) orc_weights(family, I, m, frac[a * np + p], w[a], NULL);
        for (int k = 0; k < C; ++k) {
            const double* s = stencil + (p * C + k) * I3;
            double acc = 0.0;
            for (int a3 = 0; a3 < I; ++a3)
                for (int a2 = 0; a2 < I; ++a2)
                    for (int a1 = 0; a1 < I; ++a1)
                        acc += w[0][a1] * w[1][a2] * w[2][a3] * s[(a3 * I + a2) * I + a1];
            out[k * np + p] = acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Time steppers for the tracer ODE dX/dt = u(X), Eq. (tracers).             */
/*  scheme 0, RK2 (Heun, explicit trapezoid; the paper's particle stepper is */
/*    Adams-Bashforth, RK2 is the second scheme this library offers):        */
/*      k1 = u(X), X* = X + dt k1, k2 = u(X*), X' = X + dt/2 (k1 + k2)       */
/*  schemes 1, 2, 3: ABk, k = 2, 3, 4 (multi-step Adams-Bashforth, Sec. 2.2 */
/*    and the "rhs" history of Sec. 3.3.1):                                  */
/*      X' = X + dt sum_{j<q} beta^q_j u_{n-j},  q = min(k, 1 + history),     */
/*    the textbook Adams-Bashforth weights of order q (q = 1: forward Euler, */
/*    2: 3/2, -1/2; 3: 23/12, -16/12, 5/12; 4: 55/24, -59/24, 37/24,        */
/*    -9/24): a step takes the highest order its stored history allows, so  */
/*    the first k-1 steps without history start at lower orders.  rhs holds  */
/*    k-1 entries [k-1][3][np], u_{n-1} first; `history_valid` of them are   */
/*    valid on entry; on return they hold the k-1 newest u.                  */
/* ------------------------------------------------------------------------ */
/* Adams-Bashforth weights by order q (row q - 1), newest rhs first */
static const double AB_BETA[4][4] = {
    { 1.0, 0.0, 0.0, 0.0 },
    { 3.0 / 2.0, -1.0 / 2.0, 0.0, 0.0 },
    { 23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0, 0.0 },
    { 55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0 },
};

static int eval_u(const struct orc_kernel* K, const double* f, int N, double inv_delta,
                  const double X[3], double u[3])
{
    int32_t c[3]; double t[3];
    for (int a = 0; a < 3; ++a) if (split_one(X[a], N, inv_delta, &c[a], &t[a])) return -1;
    interp_one(K, f, 3, N, inv_delta, c, t, 0, u);
    return 0;
}

static int eval_J(const struct orc_kernel* K, const double* f, int N, double inv_delta,
                  const double X[3], double J[9] /* J[k*3+j] = du_k/dX_j */)
{
    int32_t c[3]; double t[3];
    for (int a = 0; a < 3; ++a) if (split_one(X[a], N, inv_delta, &c[a], &t[a])) return -1;
    interp_one(K, f, 3, N, inv_delta, c, t, 1, J);
    return 0;
}

int orc_advance(int family, int I, int m, int N, double L, const double* field,
                int64_t np, double* pos, double* rhs, double dt, int steps, int scheme, int history_valid)
{
    struct orc_kernel K = { family, I, m };
    if (orc_check_kernel(family, I, m)) return -1;
    if (scheme < 0 || scheme > 3) return -1;
    const int k = scheme == 0 ? 0 : scheme + 1;          /* AB order */
    if (k && !rhs) return -1;
    if (k && (history_valid < 0 || history_valid > k - 1)) return -1;
    double inv_delta = orc_inv_delta(N, L);
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(|:bad)
    for (int64_t p = 0; p < np; ++p) {
        double X[3] = { pos[p], pos[np + p], pos[2 * np + p] };
        double H[3][3] = { { 0 } };                     /* H[e][a] = u_{n-1-e}, axis a */
        int hv = history_valid;
        for (int e = 0; e < k - 1; ++e)
            for (int a = 0; a < 3; ++a) H[e][a] = rhs[((int64_t)e * 3 + a) * np + p];
        for (int s = 0; s < steps; ++s) {
            double k1[3];
            if (eval_u(&K, field, N, inv_delta, X, k1)) { bad = 1; break; }
            if (scheme == 0) {
                double Xs[3], k2[3];
                for (int a = 0; a < 3; ++a) Xs[a] = X[a] + dt * k1[a];
                if (eval_u(&K, field, N, inv_delta, Xs, k2)) { bad = 1; break; }
                for (int a = 0; a < 3; ++a) X[a] = X[a] + 0.5 * dt * (k1[a] + k2[a]);
            } else {
                const int q = hv + 1 < k ? hv + 1 : k;
                for (int a = 0; a < 3; ++a) {
                    double inc = AB_BETA[q - 1][0] * k1[a];
                    for (int j = 1; j < q; ++j) inc += AB_BETA[q - 1][j] * H[j - 1][a];
                    X[a] = X[a] + dt * inc;
                }
                for (int e = k - 2; e > 0; --e)
                    for (int a = 0; a < 3; ++a) H[e][a] = H[e - 1][a];
                for (int a = 0; a < 3; ++a) H[0][a] = k1[a];
                if (hv < k - 1) ++hv;
            }
        }
        for (int a = 0; a < 3; ++a) pos[a * np + p] = X[a];
        for (int e = 0; e < k - 1; ++e)
            for (int a = 0; a < 3; ++a) rhs[((int64_t)e * 3 + a) * np + p] = H[e][a];
    }
    return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of `steps` RK2 (Heun) steps, 3-component field.          */
/* Given lambda = dLoss/dX_T, returns dLoss/dX_0 and accumulates             */
/* dLoss/dfield.  Per step, backwards, with J = du/dX and W(X) the linear    */
/* map field -> u(X) (weights beta x beta x beta):                           */
/*   lambda* = dt/2 J(X*)^T lambda                                          */
/*   mu      = dt/2 lambda + dt lambda*                                      */
/*   gfield += W(X)^T mu + W(X*)^T (dt/2 lambda)                             */
/*   lambda <- lambda + lambda* + J(X)^T mu                                  */
/* All intermediate states are stored (checkpointing only changes memory,    */
/* not the result).  Particles are independent except for the shared field   */
/* gradient, which is summed serially in particle order.                     */
/* ------------------------------------------------------------------------ */
static void scatter_W(const struct orc_kernel* K, int N, double inv_delta, const double X[3],
                      const double mu[3], double* gfield)
{
    int32_t c[3]; double t[3];
    for (int a = 0; a < 3; ++a) split_one(X[a], N, inv_delta, &c[a], &t[a]);
    int I = K->I;
    double w[3][ORC_MAX_I];
    for (int a = 0; a < 3; ++a) orc_weights(K->family, I, K->m, t[a], w[a], NULL);
    int lo = 1 - I / 2;
    int64_t NN = N;
    for (int a3 = 0; a3 < I; ++a3) {
        int64_t x3 = ((c[2] + lo + a3) % N + N) % N;
        for (int a2 = 0; a2 < I; ++a2) {
            int64_t x2 = ((c[1] + lo + a2) % N + N) % N;
            for (int a1 = 0; a1 < I; ++a1) {
                int64_t x1 = ((c[0] + lo + a1) % N + N) % N;
                int64_t node = (x3 * NN + x2) * NN + x1;
                double wt = w[0][a1] * w[1][a2] * w[2][a3];
                for (int k = 0; k < 3; ++k) gfield[(int64_t)k * NN * NN * NN + node] += wt * mu[k];
            }
        }
    }
}

int orc_adjoint_rk2(int family, int I, int m, int N, double L, const double* field,
                    int64_t np, const double* pos0, const double* lambdaT, double dt, int steps,
                    double* grad_pos0, double* grad_field /* [3][N^3], accumulated into */)
{
    struct orc_kernel K = { family, I, m };
    if (orc_check_kernel(family, I, m)) return -1;
    double inv_delta = orc_inv_delta(N, L);
    double* traj = (double*)malloc((size_t)(steps + 1) * 3 * (size_t)np * sizeof(double));
    if (!traj) return -2;
    /* forward, storing every state: traj[s][a][p] */
    memcpy(traj, pos0, 3 * (size_t)np * sizeof(double));
    for (int s = 0; s < steps; ++s) {
        memcpy(traj + (size_t)(s + 1) * 3 * np, traj + (size_t)s * 3 * np, 3 * (size_t)np * sizeof(double));
        int rc = orc_advance(family, I, m, N, L, field, np, traj + (size_t)(s + 1) * 3 * np, NULL, dt, 1, 0, 0);
        if (rc) { free(traj); return rc; }
    }
    memcpy(grad_pos0, lambdaT, 3 * (size_t)np * sizeof(double));
    for (int s = steps - 1; s >= 0; --s) {
        const double* Xs = traj + (size_t)s * 3 * np;
        for (int64_t p = 0; p < np; ++p) {
            double X[3] = { Xs[p], Xs[np + p], Xs[2 * np + p] };
            double lam[3] = { grad_pos0[p], grad_pos0[np + p], grad_pos0[2 * np + p] };
            double k1[3], J1[9], J2[9], Xst[3];
            if (eval_u(&K, field, N, inv_delta, X, k1)) { free(traj); return -4; }
            for (int a = 0; a < 3; ++a) Xst[a] = X[a] + dt * k1[a];
            eval_J(&K, field, N, inv_delta, X, J1);
            eval_J(&K, field, N, inv_delta, Xst, J2);
            double lst[3], mu[3], half[3];
            for (int j = 0; j < 3; ++j) {
                double s2 = 0.0;
                for (int k = 0; k < 3; ++k) s2 += J2[k * 3 + j] * lam[k];
                lst[j] = 0.5 * dt * s2;
            }
            for (int k = 0; k < 3; ++k) { mu[k] = 0.5 * dt * lam[k] + dt * lst[k]; half[k] = 0.5 * dt * lam[k]; }
            if (grad_field) {
                scatter_W(&K, N, inv_delta, X, mu, grad_field);
                scatter_W(&K, N, inv_delta, Xst, half, grad_field);
            }
            for (int j = 0; j < 3; ++j) {
                double s1 = 0.0;
                for (int k = 0; k < 3; ++k) s1 += J1[k * 3 + j] * mu[k];
                grad_pos0[j * np + p] = lam[j] + lst[j] + s1;
            }
        }
    }
    free(traj);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
