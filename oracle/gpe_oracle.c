/*
 * gpe_oracle.c -- plain FP64 CPU oracle for the finite-difference
 * Gross-Pitaevskii (GPE) step on a selectively sampled Cartesian grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this
 * code: it exists so that tests, the smoke check and the CPU baseline of
 * the benchmark can compare the CUDA library against an obviously correct
 * restatement of the method.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * Paper: "Efficient simulation of Bose-Einstein condensates in nontrivial
 * topologies" (Beregi, Gerent, Lundblad).  Units hbar = m = 1.
 *
 * Discrete problem (Sec. II A, general algorithm):
 *   - a Cartesian box nx*ny*nz with spacings hx, hy, hz; cell (i,j,k) has
 *     linear index  i + nx*(j + ny*k)  (x fastest);
 *   - the region of interest is an explicit list of active cells, given in
 *     ascending linear order;  rows and columns of every other cell are
 *     deleted from the Kronecker-sum 7-point Laplacian, i.e. psi == 0 there
 *     and those cells are never updated (Dirichlet zero);
 *   - T = -1/2 * Laplacian (the kinetic operator, including its prefactor).
 *
 * Everything is plain loops over the active-cell list; OpenMP is used only
 * to split independent cells between threads.  Complex numbers use C99
 * "double complex", laid out as (re, im) pairs of doubles.
 *
 * Pins (what keeps this file honest) live in tests/test_oracle_pins.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* direction order used by the neighbour table: -x, +x, -y, +y, -z, +z */

/* ------------------------------------------------------------------ */
/* Neighbour lookup: independent of any GPU layout.  For every active   */
/* cell and each of the six face directions, find the position of the   */
/* neighbouring cell in the (sorted) active list by binary search, or   */
/* -1 when the neighbour is outside the box or not active.              */
/* ------------------------------------------------------------------ */
static int64_t find_cell(int64_t n, const int64_t *cells, int64_t key)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cells[mid] == key) return mid;
        if (cells[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int orc_neighbors(int64_t n, const int64_t *cells, int64_t nx, int64_t ny,
                  int64_t nz, int64_t *nbr)
{
    for (int64_t c = 1; c < n; ++c)
        if (cells[c] <= cells[c - 1]) return -1;   /* must be ascending */
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        int64_t lin = cells[c];
        int64_t i = lin % nx, j = (lin / nx) % ny, k = lin / (nx * ny);
        int64_t d[6][3] = {{-1,0,0},{1,0,0},{0,-1,0},{0,1,0},{0,0,-1},{0,0,1}};
        for (int e = 0; e < 6; ++e) {
            int64_t ii = i + d[e][0], jj = j + d[e][1], kk = k + d[e][2];
            int64_t r = -1;
            if (ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz)
                r = find_cell(n, cells, ii + nx * (jj + ny * kk));
            nbr[6 * c + e] = r;
        }
    }
    return 0;
}

static inline cplx val(const cplx *psi, int64_t idx)
{
    return idx < 0 ? 0.0 : psi[idx];
}

/* ------------------------------------------------------------------ */
/* 7-point Laplacian (Sec. II A; Eq. (B1) of App. B for unequal         */
/* spacings):  sum over axes of (psi[+e] - 2 psi + psi[-e]) / h_e^2,    */
/* with absent neighbours contributing zero.                            */
/* ------------------------------------------------------------------ */
void orc_laplacian(int64_t n, const int64_t *nbr, double hx, double hy,
                   double hz, const cplx *psi, cplx *out)
{
    double ih2[3] = {1.0 / (hx * hx), 1.0 / (hy * hy), 1.0 / (hz * hz)};
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        cplx s = 0.0;
        for (int a = 0; a < 3; ++a) {
            cplx lo = val(psi, nbr[6 * c + 2 * a]);
            cplx hi = val(psi, nbr[6 * c + 2 * a + 1]);
            s += (hi - 2.0 * psi[c] + lo) * ih2[a];
        }
        out[c] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Edge neighbours for the 19-point stencil: for every active cell the  */
/* 12 cells that differ by one step along two axes, in the order        */
/* xy: (-1,-1,0) (+1,-1,0) (-1,+1,0) (+1,+1,0);                         */
/* xz: (-1,0,-1) (+1,0,-1) (-1,0,+1) (+1,0,+1);                         */
/* yz: (0,-1,-1) (0,+1,-1) (0,-1,+1) (0,+1,+1);  -1 when absent.        */
/* ------------------------------------------------------------------ */
int orc_edge_neighbors(int64_t n, const int64_t *cells, int64_t nx, int64_t ny,
                       int64_t nz, int64_t *nbr_e)
{
    static const int64_t d[12][3] = {{-1,-1,0},{1,-1,0},{-1,1,0},{1,1,0},
                                     {-1,0,-1},{1,0,-1},{-1,0,1},{1,0,1},
                                     {0,-1,-1},{0,1,-1},{0,-1,1},{0,1,1}};
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        int64_t lin = cells[c];
        int64_t i = lin % nx, j = (lin / nx) % ny, k = lin / (nx * ny);
        for (int e = 0; e < 12; ++e) {
            int64_t ii = i + d[e][0], jj = j + d[e][1], kk = k + d[e][2];
            int64_t r = -1;
            if (ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz)
                r = find_cell(n, cells, ii + nx * (jj + ny * kk));
            nbr_e[12 * c + e] = r;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 19-point higher-order compact Laplacian for unequal spacings (App. B):*/
/*   L19 = L7 + 1/12 [ (hx^2+hy^2) dx2 dy2 + (hx^2+hz^2) dx2 dz2         */
/*                    + (hy^2+hz^2) dy2 dz2 ],                           */
/* dx2 dy2 psi = (sum of the 4 xy-edge cells - 2 (sum of the 4 xy face  */
/* cells) + 4 psi) / (hx^2 hy^2), and likewise for xz and yz.            */
/* ------------------------------------------------------------------ */
void orc_laplacian19(int64_t n, const int64_t *nbr, const int64_t *nbr_e, double hx,
                     double hy, double hz, const cplx *psi, cplx *out)
{
    const double h2[3] = {hx * hx, hy * hy, hz * hz};
    orc_laplacian(n, nbr, hx, hy, hz, psi, out);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        cplx mixed = 0.0;
        for (int p = 0; p < 3; ++p) {            /* planes xy, xz, yz */
            const int a = p == 2 ? 1 : 0;        /* first axis of the plane */
            const int b = p == 0 ? 1 : 2;        /* second axis */
            cplx edges = 0.0;
            for (int q = 0; q < 4; ++q) edges += val(psi, nbr_e[12 * c + 4 * p + q]);
            cplx faces = val(psi, nbr[6 * c + 2 * a]) + val(psi, nbr[6 * c + 2 * a + 1]) +
                         val(psi, nbr[6 * c + 2 * b]) + val(psi, nbr[6 * c + 2 * b + 1]);
            cplx d2d2 = (edges - 2.0 * faces + 4.0 * psi[c]) / (h2[a] * h2[b]);
            mixed += (h2[a] + h2[b]) * d2d2;
        }
        out[c] += mixed / 12.0;
    }
}

/* H psi = (T + V + g|psi|^2) psi with T = -1/2 Laplacian (Eq. (2)). */
static void apply_H(int64_t n, const int64_t *nbr, const double h[3],
                    const double *V, double g, const cplx *psi, cplx *out)
{
    orc_laplacian(n, nbr, h[0], h[1], h[2], psi, out);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        double rho = creal(psi[c]) * creal(psi[c]) + cimag(psi[c]) * cimag(psi[c]);
        out[c] = -0.5 * out[c] + (V[c] + g * rho) * psi[c];
    }
}

/* ------------------------------------------------------------------ */
/* Time-dependent potential used by the ramp: V(t) = (1-s)V0 + s V1,   */
/* with s(t) piecewise linear through n_knots values placed uniformly  */
/* on [0, T] and held constant outside (the linear interpolation        */
/* between two precomputed potentials of Sec. V).                       */
/* ------------------------------------------------------------------ */
double orc_ramp_s(int n_knots, const double *knots, double T, double t)
{
    if (t <= 0.0) return knots[0];
    if (t >= T) return knots[n_knots - 1];
    double u = t / T * (double)(n_knots - 1);
    int k = (int)floor(u);
    if (k >= n_knots - 1) k = n_knots - 2;
    double w = u - (double)k;
    return (1.0 - w) * knots[k] + w * knots[k + 1];
}

/* weight of knot q in s(t): the hat function of the interpolation */
static double ramp_hat(int n_knots, double T, double t, int q)
{
    if (t <= 0.0) return q == 0 ? 1.0 : 0.0;
    if (t >= T) return q == n_knots - 1 ? 1.0 : 0.0;
    double u = t / T * (double)(n_knots - 1);
    int k = (int)floor(u);
    if (k >= n_knots - 1) k = n_knots - 2;
    double w = u - (double)k;
    if (q == k) return 1.0 - w;
    if (q == k + 1) return w;
    return 0.0;
}

static void potential_at(int64_t n, const double *V0, const double *V1,
                         int n_knots, const double *knots, double T, double t,
                         double *Vt)
{
    double s = (V1 && n_knots > 0) ? orc_ramp_s(n_knots, knots, T, t) : 0.0;
    for (int64_t c = 0; c < n; ++c)
        Vt[c] = (V1 && n_knots > 0) ? (1.0 - s) * V0[c] + s * V1[c] : V0[c];
}

/* Right-hand side of the real-time equation (Eq. (8)):
 * f(t, y) = -i (T + V(t) + g|y|^2) y.                                   */
void orc_rhs_real(int64_t n, const int64_t *nbr, double hx, double hy,
                  double hz, const double *V, double g, const cplx *y,
                  cplx *f)
{
    double h[3] = {hx, hy, hz};
    apply_H(n, nbr, h, V, g, y, f);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) f[c] = -I * f[c];
}

/* ------------------------------------------------------------------ */
/* Classic fourth-order Runge-Kutta step (Sec. II A, RK4), written in   */
/* the standard Butcher form k1..k4 of Eq. (9): stage i evaluates f at  */
/* t + c_i dt with c = (0, 1/2, 1/2, 1) and                             */
/* y1 = y0 + dt (k1 + 2 k2 + 2 k3 + k4) / 6.                            */
/* V1 == NULL (or n_knots == 0) means a static potential V0.            */
/* ------------------------------------------------------------------ */
int orc_rk4_step(int64_t n, const int64_t *nbr, double hx, double hy,
                 double hz, const double *V0, const double *V1, int n_knots,
                 const double *knots, double T, double g, double t, double dt,
                 cplx *y)
{
    cplx *k1 = malloc(sizeof(cplx) * (size_t)n), *k2 = malloc(sizeof(cplx) * (size_t)n);
    cplx *k3 = malloc(sizeof(cplx) * (size_t)n), *k4 = malloc(sizeof(cplx) * (size_t)n);
    cplx *ys = malloc(sizeof(cplx) * (size_t)n);
    double *Vt = malloc(sizeof(double) * (size_t)n);
    if (!k1 || !k2 || !k3 || !k4 || !ys || !Vt) {
        free(k1); free(k2); free(k3); free(k4); free(ys); free(Vt);
        return -1;
    }
    const double c[4] = {0.0, 0.5, 0.5, 1.0};
    cplx *k[4] = {k1, k2, k3, k4};
    for (int s = 0; s < 4; ++s) {
        /* stage state y^(s) = y0 + dt * a_{s,s-1} k_{s-1}  (RK4 is explicit
         * with only the sub-diagonal of its tableau non-zero)            */
        const double a_prev[4] = {0.0, 0.5, 0.5, 1.0};
        for (int64_t q = 0; q < n; ++q)
            ys[q] = (s == 0) ? y[q] : y[q] + dt * a_prev[s] * k[s - 1][q];
        potential_at(n, V0, V1, n_knots, knots, T, t + c[s] * dt, Vt);
        orc_rhs_real(n, nbr, hx, hy, hz, Vt, g, ys, k[s]);
    }
    for (int64_t q = 0; q < n; ++q)
        y[q] += dt / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
    free(k1); free(k2); free(k3); free(k4); free(ys); free(Vt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* General explicit Runge-Kutta step in Butcher form (the integrators   */
/* whose memory-optimised forms App. A tabulates: RKHE3, RK4, RKCK):    */
/*   k_i = f(t + c_i dt, y0 + dt sum_{j<i} A_ij k_j),  i = 1..s,        */
/*   y1  = y0 + dt sum_i b_i k_i.                                       */
/* A is s x s, row-major, only its strictly lower part is read.         */
/* ------------------------------------------------------------------ */
int orc_rk_step(int64_t n, const int64_t *nbr, double hx, double hy,
                double hz, const double *V0, const double *V1, int n_knots,
                const double *knots, double T, double g, double t, double dt,
                int s, const double *A, const double *b, const double *c,
                cplx *y)
{
    if (s < 1 || s > 16) return -2;
    cplx *k = malloc(sizeof(cplx) * (size_t)n * (size_t)s);
    cplx *ys = malloc(sizeof(cplx) * (size_t)n);
    double *Vt = malloc(sizeof(double) * (size_t)n);
    if (!k || !ys || !Vt) {
        free(k); free(ys); free(Vt);
        return -1;
    }
    for (int i = 0; i < s; ++i) {
        for (int64_t q = 0; q < n; ++q) {
            cplx acc = 0.0;
            for (int j = 0; j < i; ++j) acc += A[i * s + j] * k[(size_t)j * n + q];
            ys[q] = y[q] + dt * acc;
        }
        potential_at(n, V0, V1, n_knots, knots, T, t + c[i] * dt, Vt);
        orc_rhs_real(n, nbr, hx, hy, hz, Vt, g, ys, k + (size_t)i * n);
    }
    for (int64_t q = 0; q < n; ++q) {
        cplx acc = 0.0;
        for (int i = 0; i < s; ++i) acc += b[i] * k[(size_t)i * n + q];
        y[q] += dt * acc;
    }
    free(k); free(ys); free(Vt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Imaginary-time step (Sec. II A, Eq. (6), Eq. (7) and the text after  */
/* it), in the paper's order:                                           */
/*   1. diagonal half step  psi <- psi * exp(-V dt/2) * (1 - g|psi|^2 dt/2) */
/*      (interaction propagator linearised, |psi|^2 of the input psi);  */
/*   2. kinetic propagation over dt in two forward-Euler substeps of    */
/*      dt/2 each: psi <- psi - (dt/2) T psi, twice;                    */
/*   3. the diagonal half step again;                                   */
/*   4. renormalise to N:  psi <- psi * sqrt(N / (sum |psi|^2 dV)).     */
/* Returns the norm sum|psi|^2 dV measured before step 4.               */
/* ------------------------------------------------------------------ */
double orc_itp_step(int64_t n, const int64_t *nbr, double hx, double hy,
                    double hz, const double *V, double g, double dt, double N,
                    cplx *psi)
{
    cplx *lap = malloc(sizeof(cplx) * (size_t)n);
    if (!lap) return -1.0;
    for (int half = 0; half < 2; ++half) {
        if (half == 1) {
            for (int sub = 0; sub < 2; ++sub) {
                orc_laplacian(n, nbr, hx, hy, hz, psi, lap);
                for (int64_t c = 0; c < n; ++c)
                    psi[c] = psi[c] - 0.5 * dt * (-0.5 * lap[c]);
            }
        }
        for (int64_t c = 0; c < n; ++c) {
            double rho = creal(psi[c]) * creal(psi[c]) + cimag(psi[c]) * cimag(psi[c]);
            psi[c] = psi[c] * exp(-V[c] * dt / 2.0) * (1.0 - g * rho * dt / 2.0);
        }
    }
    free(lap);
    double dV = hx * hy * hz, norm = 0.0;
    for (int64_t c = 0; c < n; ++c)
        norm += (creal(psi[c]) * creal(psi[c]) + cimag(psi[c]) * cimag(psi[c])) * dV;
    double s = sqrt(N / norm);
    for (int64_t c = 0; c < n; ++c) psi[c] *= s;
    return norm;
}

/* ------------------------------------------------------------------ */
/* Observables with the discrete operator:                              */
/*   norm = sum |psi|^2 dV                        (Eq. (3))            */
/*   E    = sum dV [Re(conj(psi) T psi) + V|psi|^2 + (g/2)|psi|^4]      */
/*   mu   = sum dV [Re(conj(psi) T psi) + V|psi|^2 + g|psi|^4] / norm   */
/*          (the GP energy functional whose variation gives Eq. (1))    */
/*   nonfinite = number of cells whose value is NaN or infinite.        */
/* out = {norm, E, mu, nonfinite, E_kin, E_pot, E_int}                  */
/* ------------------------------------------------------------------ */
void orc_observables(int64_t n, const int64_t *nbr, double hx, double hy,
                     double hz, const double *V, double g, const cplx *psi,
                     double *out)
{
    cplx *lap = malloc(sizeof(cplx) * (size_t)n);
    orc_laplacian(n, nbr, hx, hy, hz, psi, lap);
    double dV = hx * hy * hz;
    double nrm = 0.0, ekin = 0.0, epot = 0.0, eint = 0.0, bad = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        double rho = creal(psi[c]) * creal(psi[c]) + cimag(psi[c]) * cimag(psi[c]);
        if (!isfinite(creal(psi[c])) || !isfinite(cimag(psi[c]))) bad += 1.0;
        nrm += rho * dV;
        ekin += creal(conj(psi[c]) * (-0.5 * lap[c])) * dV;
        epot += V[c] * rho * dV;
        eint += 0.5 * g * rho * rho * dV;
    }
    free(lap);
    out[0] = nrm;
    out[1] = ekin + epot + eint;
    out[2] = (ekin + epot + 2.0 * eint) / nrm;
    out[3] = bad;
    out[4] = ekin;
    out[5] = epot;
    out[6] = eint;
}

/* <a|b> = sum conj(a) b dV */
void orc_overlap(int64_t n, const cplx *a, const cplx *b, double dV, double *out)
{
    cplx s = 0.0;
    for (int64_t c = 0; c < n; ++c) s += conj(a[c]) * b[c];
    out[0] = creal(s) * dV;
    out[1] = cimag(s) * dV;
}

/* ------------------------------------------------------------------ */
/* Thomas-Fermi chemical potential (Sec. II A, Eq. (5)): the mu for     */
/* which sum max((mu - V)/g, 0) dV equals N, found by bisection on mu   */
/* (the paper adjusts mu until the trial atom number is the one wanted).*/
/* ------------------------------------------------------------------ */
static double tf_number(int64_t n, const double *V, double dV, double g, double mu)
{
    double s = 0.0;
    for (int64_t c = 0; c < n; ++c)
        if (mu > V[c]) s += (mu - V[c]) / g * dV;
    return s;
}

double orc_tf_mu(int64_t n, const double *V, double dV, double g, double N)
{
    double lo = V[0], hi = V[0];
    for (int64_t c = 1; c < n; ++c) {
        if (V[c] < lo) lo = V[c];
        if (V[c] > hi) hi = V[c];
    }
    /* grow the upper bracket until it holds at least N atoms */
    double span = (hi - lo) > 0 ? (hi - lo) : 1.0;
    while (tf_number(n, V, dV, g, hi) < N) hi += span, span *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (tf_number(n, V, dV, g, mid) < N) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of one Butcher-form RK4 step (orc_rk4_step).        */
/*                                                                      */
/* psi is treated as the real pair (Re, Im); a gradient is stored as    */
/* the complex number dL/dRe + i dL/dIm.  For the right-hand side       */
/*   f(y) = -i [ (T + V) y + g |y|^2 y ]                                 */
/* the transposed Jacobian acting on a gradient G is                    */
/*   J^T G = i (T + V) G + 2 i g |y|^2 G - i g y^2 conj(G)              */
/* (T and V are real symmetric).  Reversing the four stages:            */
/*   mu4 = dt/6 lam' ;            nu4 = J4^T mu4                        */
/*   mu3 = dt/3 lam' + dt nu4 ;   nu3 = J3^T mu3                        */
/*   mu2 = dt/3 lam' + dt/2 nu3 ; nu2 = J2^T mu2                        */
/*   mu1 = dt/6 lam' + dt/2 nu2 ; nu1 = J1^T mu1                        */
/*   lam = lam' + nu1 + nu2 + nu3 + nu4                                  */
/* and every stage adds Re<mu_i, -i (V1 - V0) Y_i> times the hat weight  */
/* of each knot at t + c_i dt to the knot gradient.                     */
/* y0 is the state at the START of the step (unchanged); lam holds      */
/* dL/dy1 on entry and dL/dy0 on return; grad (n_knots) is accumulated. */
/* ------------------------------------------------------------------ */
static void apply_JT(int64_t n, const int64_t *nbr, const double h[3],
                     const double *Vt, double g, const cplx *Y, const cplx *G,
                     cplx *out)
{
    orc_laplacian(n, nbr, h[0], h[1], h[2], G, out);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        double rho = creal(Y[c]) * creal(Y[c]) + cimag(Y[c]) * cimag(Y[c]);
        cplx TG = -0.5 * out[c];
        out[c] = I * (TG + Vt[c] * G[c]) + 2.0 * I * g * rho * G[c]
               - I * g * Y[c] * Y[c] * conj(G[c]);
    }
}

int orc_rk4_adjoint_step(int64_t n, const int64_t *nbr, double hx, double hy,
                         double hz, const double *V0, const double *V1,
                         int n_knots, const double *knots, double T, double g,
                         double t, double dt, const cplx *y0, cplx *lam,
                         double *grad)
{
    double h[3] = {hx, hy, hz};
    const double c[4] = {0.0, 0.5, 0.5, 1.0};
    const double a_prev[4] = {0.0, 0.5, 0.5, 1.0};
    size_t bytes = sizeof(cplx) * (size_t)n;
    cplx *Y[4], *k = malloc(bytes), *mu = malloc(bytes), *nu = malloc(bytes);
    cplx *acc = malloc(bytes);
    double *Vt = malloc(sizeof(double) * (size_t)n);
    for (int s = 0; s < 4; ++s) Y[s] = malloc(bytes);
    /* forward recomputation of the stage states Y1..Y4 */
    for (int s = 0; s < 4; ++s) {
        for (int64_t q = 0; q < n; ++q)
            Y[s][q] = (s == 0) ? y0[q] : y0[q] + dt * a_prev[s] * k[q];
        potential_at(n, V0, V1, n_knots, knots, T, t + c[s] * dt, Vt);
        orc_rhs_real(n, nbr, hx, hy, hz, Vt, g, Y[s], k);
    }
    /* reverse sweep */
    const double w_b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int64_t q = 0; q < n; ++q) acc[q] = lam[q];
    for (int s = 3; s >= 0; --s) {
        for (int64_t q = 0; q < n; ++q) {
            mu[q] = dt * w_b[s] * lam[q];
            if (s < 3) mu[q] += dt * a_prev[s + 1] * nu[q];
        }
        double ts = t + c[s] * dt;
        if (V1 && n_knots > 0 && grad) {
            double dot = 0.0;   /* Re <mu, -i (V1 - V0) Y> */
            for (int64_t q = 0; q < n; ++q)
                dot += creal(conj(mu[q]) * (-I * (V1[q] - V0[q]) * Y[s][q]));
            for (int kk = 0; kk < n_knots; ++kk)
                grad[kk] += ramp_hat(n_knots, T, ts, kk) * dot;
        }
        potential_at(n, V0, V1, n_knots, knots, T, ts, Vt);
        apply_JT(n, nbr, h, Vt, g, Y[s], mu, nu);
        for (int64_t q = 0; q < n; ++q) acc[q] += nu[q];
    }
    for (int64_t q = 0; q < n; ++q) lam[q] = acc[q];
    for (int s = 0; s < 4; ++s) free(Y[s]);
    free(k); free(mu); free(nu); free(acc); free(Vt);
    return 0;
}
