/*
 * lgf_oracle.c -- plain FP64 CPU oracle for Fourier-accelerated steepest-descent
 * Landau gauge fixing of a 4D SU(3) lattice gauge field (Cardoso, Silva,
 * Oliveira, Bicudo, "Landau gauge fixing on the lattice using GPU's",
 * arXiv:1301.3460).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against and the timed CPU baseline.  Only the test
 * suite, the smoke entry point and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant with the CUDA path.
 *
 * What the paper fixes and what is read into it:
 *   - The functional (display equation of the introduction):
 *       F_U[g] = 1/(N_d N_c V) sum_x sum_mu Re Tr[g(x) U_mu(x) g^dag(x+mu)].
 *     F of the current links is F with g = 1.
 *   - The maximisation is steepest descent with Fourier acceleration
 *     (introduction, citing Davies et al. and Oliveira-Silva); the run
 *     parameters alpha = 0.08 and the stop at theta < 1e-15 are given in the
 *     description of the 32^4 comparison.
 *   - The paper does not write out Delta, theta, the accelerator, the
 *     exponentiation or the reunitarisation.  The readings used here are the
 *     standard ones of the cited steepest-descent literature:
 *       M(x)     = sum_mu [ U_mu(x-mu) - U_mu(x) ]
 *       Delta(x) = (M - M^dag) - (1/3) Tr(M - M^dag) 1      (traceless anti-Hermitian)
 *       theta    = 1/(N_c V) sum_x Tr[Delta Delta^dag]
 *       Delta~   = IDFT[ p2max/p2(k) * DFT[Delta](k) ] / V,  k = 0 mode removed,
 *                  p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu),  p2max = max_k p2(k)
 *       g(x)     = reunit(1 + (alpha/2) Delta~(x))           (row Gram-Schmidt)
 *       U_mu(x) <- g(x) U_mu(x) g^dag(x+mu),  G(x) <- g(x) G(x)
 *     Rows 0,1 carry the link (the 12-real link storage of the paper's GPU
 *     code); row 2 is recomputed as conj(row0 x row1) after every
 *     update, for links and for the accumulated gauge transformation G.
 *
 * Storage: a link field is [4][V][3][3] complex double (mu-major, then site,
 * then row, column); a site field of matrices is [V][3][3]; a scalar field is
 * [V].  Site index s = x + Lx*(y + Ly*(z + Lz*t)).
 *
 * The FFT is a recursive mixed-radix decimation-in-time transform applied along
 * each axis; the direct DFT is the O(V^2) definition and is used on tiny
 * lattices and to pin the FFT.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define NC 3
#define ND 4

/* ------------------------------------------------------------------ */
/* lattice geometry                                                     */
/* ------------------------------------------------------------------ */

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long s, int c[4])
{
    for (int mu = 0; mu < 4; mu++) { c[mu] = (int)(s % L[mu]); s /= L[mu]; }
}

static long site(const int L[4], const int c[4])
{
    long s = 0;
    for (int mu = 3; mu >= 0; mu--) s = s * L[mu] + c[mu];
    return s;
}

/* site shifted by d (+1 or -1) along mu, periodic */
static long shift(const int L[4], long s, int mu, int d)
{
    int c[4];
    coords(L, s, c);
    c[mu] = (c[mu] + d + L[mu]) % L[mu];
    return site(L, c);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* 3x3 complex matrices, row-major                                      */
/* ------------------------------------------------------------------ */

static void mat_mul(const cplx* a, const cplx* b, cplx* c) /* c = a b */
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += a[3 * i + k] * b[3 * k + j];
            t[3 * i + j] = acc;
        }
    memcpy(c, t, sizeof t);
}

static void mat_mul_dag(const cplx* a, const cplx* b, cplx* c) /* c = a b^dag */
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += a[3 * i + k] * conj(b[3 * j + k]);
            t[3 * i + j] = acc;
        }
    memcpy(c, t, sizeof t);
}

/* row 2 := conj(row0 x row1): the SU(3) completion of two orthonormal rows */
static void complete_row2(cplx* m)
{
    const cplx* r0 = m;
    const cplx* r1 = m + 3;
    m[6] = conj(r0[1] * r1[2] - r0[2] * r1[1]);
    m[7] = conj(r0[2] * r1[0] - r0[0] * r1[2]);
    m[8] = conj(r0[0] * r1[1] - r0[1] * r1[0]);
}

/* Row Gram-Schmidt projection onto SU(3):
 *   r0 = X0/|X0|,  r1 = (X1 - <r0,X1> r0)/|.|,  r2 = conj(r0 x r1),
 * with <a,b> = sum_j conj(a_j) b_j. */
void orc_reunit(const cplx* X, cplx* g)
{
    cplx r[9];
    double n0 = 0;
    for (int j = 0; j < 3; j++) n0 += creal(X[j] * conj(X[j]));
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; j++) r[j] = X[j] * n0;
    cplx ip = 0;
    for (int j = 0; j < 3; j++) ip += conj(r[j]) * X[3 + j];
    double n1 = 0;
    for (int j = 0; j < 3; j++) {
        r[3 + j] = X[3 + j] - ip * r[j];
        n1 += creal(r[3 + j] * conj(r[3 + j]));
    }
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; j++) r[3 + j] *= n1;
    complete_row2(r);
    memcpy(g, r, sizeof r);
}

/* ------------------------------------------------------------------ */
/* Delta, theta, F                                                      */
/* ------------------------------------------------------------------ */

/* Delta(x) for every site, theta and F of the links U.  Delta may be NULL. */
void orc_delta(const int L[4], const cplx* U, cplx* Delta, double* theta, double* F)
{
    const long V = volume(L);
    double th = 0, f = 0;
#pragma omp parallel for schedule(static) reduction(+ : th, f)
    for (long s = 0; s < V; s++) {
        cplx M[9] = {0};
        for (int mu = 0; mu < ND; mu++) {
            const cplx* Ub = U + ((long)mu * V + shift(L, s, mu, -1)) * 9; /* U_mu(x-mu) */
            const cplx* Uf = U + ((long)mu * V + s) * 9;                   /* U_mu(x)    */
            for (int e = 0; e < 9; e++) M[e] += Ub[e] - Uf[e];
            f += creal(Uf[0] + Uf[4] + Uf[8]);
        }
        cplx D[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) D[3 * i + j] = M[3 * i + j] - conj(M[3 * j + i]);
        cplx tr = (D[0] + D[4] + D[8]) / 3.0;
        D[0] -= tr;
        D[4] -= tr;
        D[8] -= tr;
        for (int e = 0; e < 9; e++) th += creal(D[e] * conj(D[e]));
        if (Delta) memcpy(Delta + s * 9, D, sizeof D);
    }
    if (theta) *theta = th / ((double)NC * V);
    if (F) *F = f / ((double)ND * NC * V);
}

/* ------------------------------------------------------------------ */
/* Fourier transforms                                                   */
/* ------------------------------------------------------------------ */

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

/* out[k] = sum_j in[j*is] w^(j k), w = exp(sign 2 pi i / n); out is contiguous.
 * tw[m] = exp(sign 2 pi i m / n0) for the top-level length n0; a sub-transform
 * of length n uses tw[m * (n0/n)].  scratch holds n0 elements. */
static void fft_rec(int n, int n0, const cplx* in, long is, cplx* out, const cplx* tw, cplx* scratch)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    const int p = smallest_factor(n);
    const int m = n / p;
    const int step = n0 / n; /* tw index scale for length n */
    if (p == n) {            /* prime length: the definition */
        for (int k = 0; k < n; k++) {
            cplx acc = 0;
            for (int j = 0; j < n; j++) acc += in[j * is] * tw[(long)((long)j * k % n) * step];
            scratch[k] = acc;
        }
        memcpy(out, scratch, sizeof(cplx) * n);
        return;
    }
    /* decimation in time: sub-sequence r holds in[(p j + r) is], j < m */
    for (int r = 0; r < p; r++) fft_rec(m, n0, in + r * is, is * p, out + r * m, tw, scratch);
    /* X[k + m q] = sum_r w_n^(r (k + m q)) Y_r[k] */
    for (int k = 0; k < m; k++)
        for (int q = 0; q < p; q++) {
            cplx acc = 0;
            for (int r = 0; r < p; r++) acc += out[r * m + k] * tw[(long)((long)r * (k + m * q) % n) * step];
            scratch[k + m * q] = acc;
        }
    memcpy(out, scratch, sizeof(cplx) * n);
}

static void twiddles(int n, int sign, cplx* tw)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < n; m++) tw[m] = cos(two_pi * m / n) + I * (sign * sin(two_pi * m / n));
}

/* in-place 1D FFT along every line of one axis of a scalar field */
static void fft_axis(const int L[4], cplx* f, int mu, int sign)
{
    const long V = volume(L);
    const int n = L[mu];
    long stride = 1;
    for (int nu = 0; nu < mu; nu++) stride *= L[nu];
    cplx* tw = malloc(sizeof(cplx) * n);
    twiddles(n, sign, tw);
    const long nlines = V / n;
#pragma omp parallel
    {
        cplx* line = malloc(sizeof(cplx) * n);
        cplx* scratch = malloc(sizeof(cplx) * n);
#pragma omp for schedule(static)
        for (long l = 0; l < nlines; l++) {
            /* line l: lower index a < stride, upper index b; start = a + b*stride*n */
            const long a = l % stride, b = l / stride;
            cplx* start = f + a + b * stride * n;
            fft_rec(n, n, start, stride, line, tw, scratch);
            for (int k = 0; k < n; k++) start[k * stride] = line[k];
        }
        free(line);
        free(scratch);
    }
    free(tw);
}

/* unnormalised 4D FFT of a scalar field, in place; sign -1 forward, +1 inverse */
void orc_fft4(const int L[4], cplx* f, int sign)
{
    for (int mu = 0; mu < 4; mu++) fft_axis(L, f, mu, sign);
}

/* unnormalised 4D DFT by its definition: out(k) = sum_x in(x) exp(sign 2 pi i sum_mu k_mu x_mu / L_mu) */
void orc_dft4(const int L[4], const cplx* in, cplx* out, int sign)
{
    const long V = volume(L);
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (long ks = 0; ks < V; ks++) {
        int k[4], x[4];
        coords(L, ks, k);
        cplx acc = 0;
        for (long xs = 0; xs < V; xs++) {
            coords(L, xs, x);
            /* phase as an exact rational multiple of 2 pi, reduced to [0,1) */
            double ph = 0;
            for (int mu = 0; mu < 4; mu++) ph += (double)((long)k[mu] * x[mu] % L[mu]) / L[mu];
            ph -= floor(ph);
            acc += in[xs] * (cos(two_pi * ph) + I * (sign * sin(two_pi * ph)));
        }
        out[ks] = acc;
    }
}

/* lattice momentum squared p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu) */
static double p2_of(const int L[4], const int k[4])
{
    const double pi = 3.14159265358979323846264338327950;
    double p2 = 0;
    for (int mu = 0; mu < 4; mu++) {
        double sv = sin(pi * k[mu] / L[mu]);
        p2 += 4.0 * sv * sv;
    }
    return p2;
}

double orc_p2max(const int L[4])
{
    const long V = volume(L);
    double m = 0;
    for (long s = 0; s < V; s++) {
        int k[4];
        coords(L, s, k);
        double p2 = p2_of(L, k);
        if (p2 > m) m = p2;
    }
    return m;
}

/* Fourier acceleration of a matrix field: for every entry (i,j),
 *   Dt_ij = IDFT[ p2max/p2(k) * DFT[Delta_ij](k) ] / V,  k = 0 coefficient set to 0.
 * use_dft selects the O(V^2) definition instead of the FFT. */
void orc_accelerate(const int L[4], const cplx* Delta, cplx* Dt, int use_dft)
{
    const long V = volume(L);
    const double p2max = orc_p2max(L);
    cplx* f = malloc(sizeof(cplx) * V);
    cplx* h = malloc(sizeof(cplx) * V);
    double* mult = malloc(sizeof(double) * V);
    for (long s = 0; s < V; s++) {
        int k[4];
        coords(L, s, k);
        mult[s] = (s == 0) ? 0.0 : p2max / p2_of(L, k);
    }
    for (int e = 0; e < 9; e++) {
        for (long s = 0; s < V; s++) f[s] = Delta[s * 9 + e];
        if (use_dft) {
            orc_dft4(L, f, h, -1);
            for (long s = 0; s < V; s++) h[s] *= mult[s];
            orc_dft4(L, h, f, +1);
        } else {
            orc_fft4(L, f, -1);
            for (long s = 0; s < V; s++) f[s] *= mult[s];
            orc_fft4(L, f, +1);
        }
        for (long s = 0; s < V; s++) Dt[s * 9 + e] = f[s] / (double)V;
    }
    free(f);
    free(h);
    free(mult);
}

/* ------------------------------------------------------------------ */
/* gauge transformation                                                 */
/* ------------------------------------------------------------------ */

/* g(x) = reunit(1 + (alpha/2) Dt(x)) */
void orc_build_g(const int L[4], const cplx* Dt, double alpha, cplx* g)
{
    const long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        cplx X[9];
        for (int e = 0; e < 9; e++) X[e] = 0.5 * alpha * Dt[s * 9 + e];
        X[0] += 1.0;
        X[4] += 1.0;
        X[8] += 1.0;
        orc_reunit(X, g + s * 9);
    }
}

/* U_mu(x) <- g(x) U_mu(x) g^dag(x+mu) and G(x) <- g(x) G(x), each followed by
 * row 2 := conj(row0 x row1).  G may be NULL. */
void orc_update(const int L[4], cplx* U, cplx* G, const cplx* g)
{
    const long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        for (int mu = 0; mu < ND; mu++) {
            cplx* u = U + ((long)mu * V + s) * 9;
            cplx t[9];
            mat_mul(g + s * 9, u, t);
            mat_mul_dag(t, g + shift(L, s, mu, +1) * 9, u);
            complete_row2(u);
        }
        if (G) {
            mat_mul(g + s * 9, G + s * 9, G + s * 9);
            complete_row2(G + s * 9);
        }
    }
}

/* U'_mu(x) = G(x) U_mu(x) G^dag(x+mu) for a given G (no row-2 completion) */
void orc_gauge_transform(const int L[4], const cplx* U, const cplx* G, cplx* Uout)
{
    const long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++)
        for (int mu = 0; mu < ND; mu++) {
            cplx t[9];
            mat_mul(G + s * 9, U + ((long)mu * V + s) * 9, t);
            mat_mul_dag(t, G + shift(L, s, mu, +1) * 9, Uout + ((long)mu * V + s) * 9);
        }
}

/* ------------------------------------------------------------------ */
/* the iteration                                                        */
/* ------------------------------------------------------------------ */

/* Steepest descent, Fourier-accelerated (accel = 1) or plain (accel = 0: the
 * step uses Delta itself, the unaccelerated method whose critical slowing down
 * the introduction names as the reason for Fourier acceleration).  U (in/out)
 * holds the links, G (in/out, may be NULL) accumulates the applied gauge
 * transformation.  The stop test is made on the current links before an
 * update: the run ends when theta < tol or when max_iter updates have been
 * applied.  history, if not NULL, receives (theta_n, F_n) for n = 0..iters.
 * Returns 0 if converged, 1 if not. */
int orc_fix_sd(const int L[4], cplx* U, cplx* G, double alpha, double tol, int max_iter, int use_dft, int accel,
               int* iters, double* F, double* theta, double* history)
{
    const long V = volume(L);
    cplx* D = malloc(sizeof(cplx) * 9 * V);
    cplx* Dt = malloc(sizeof(cplx) * 9 * V);
    cplx* g = malloc(sizeof(cplx) * 9 * V);
    int n = 0;
    double th = 0, f = 0;
    for (;;) {
        orc_delta(L, U, D, &th, &f);
        if (history) {
            history[2 * n] = th;
            history[2 * n + 1] = f;
        }
        if (th < tol || n >= max_iter) break;
        if (accel)
            orc_accelerate(L, D, Dt, use_dft);
        else
            memcpy(Dt, D, sizeof(cplx) * 9 * V);
        orc_build_g(L, Dt, alpha, g);
        orc_update(L, U, G, g);
        n++;
    }
    free(D);
    free(Dt);
    free(g);
    if (iters) *iters = n;
    if (F) *F = f;
    if (theta) *theta = th;
    return th < tol ? 0 : 1;
}

/* the Fourier-accelerated method */
int orc_fix(const int L[4], cplx* U, cplx* G, double alpha, double tol, int max_iter, int use_dft,
            int* iters, double* F, double* theta, double* history)
{
    return orc_fix_sd(L, U, G, alpha, tol, max_iter, use_dft, 1, iters, F, theta, history);
}

/* ------------------------------------------------------------------ */
/* observables                                                          */
/* ------------------------------------------------------------------ */

/* average plaquette (1/(6V)) sum_x sum_{mu<nu} Re Tr[U_mu(x) U_nu(x+mu) U_mu^dag(x+nu) U_nu^dag(x)] / 3 */
double orc_plaquette(const int L[4], const cplx* U)
{
    const long V = volume(L);
    double acc = 0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (long s = 0; s < V; s++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                cplx a[9], b[9];
                mat_mul(U + ((long)mu * V + s) * 9, U + ((long)nu * V + shift(L, s, mu, 1)) * 9, a);
                mat_mul_dag(a, U + ((long)mu * V + shift(L, s, nu, 1)) * 9, b);
                mat_mul_dag(b, U + ((long)nu * V + s) * 9, a);
                acc += creal(a[0] + a[4] + a[8]) / 3.0;
            }
    return acc / (6.0 * V);
}

/* Landau-gauge gluon propagator at the four smallest non-zero momenta
 * (one k_mu = 1, the others 0), averaged:
 *   A_mu(x) = (U - U^dag)/(2i) - (1/3) Tr[(U - U^dag)/(2i)]
 *   A~_mu(p) = sum_x exp(-i p.x) A_mu(x),  p_nu = 2 pi k_nu / L_nu
 *   D(p) = 2 / ((N_c^2-1)(N_d-1) V) sum_mu Tr[A~_mu(p) A~_mu(p)^dag].
 * Each of the four D(p) values is written to Dp[4] if not NULL. */
double orc_gluon_pmin(const int L[4], const cplx* U, double* Dp)
{
    const long V = volume(L);
    const double two_pi = 6.283185307179586476925286766559;
    double avg = 0;
    for (int dir = 0; dir < 4; dir++) {
        double dsum = 0;
        for (int mu = 0; mu < ND; mu++) {
            cplx At[9] = {0};
            for (long s = 0; s < V; s++) {
                int c[4];
                coords(L, s, c);
                const cplx* u = U + ((long)mu * V + s) * 9;
                cplx A[9];
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) A[3 * i + j] = (u[3 * i + j] - conj(u[3 * j + i])) / (2.0 * I);
                cplx tr = (A[0] + A[4] + A[8]) / 3.0;
                A[0] -= tr;
                A[4] -= tr;
                A[8] -= tr;
                double ph = (double)c[dir] / L[dir];
                cplx e = cos(two_pi * ph) - I * sin(two_pi * ph);
                for (int k = 0; k < 9; k++) At[k] += e * A[k];
            }
            for (int k = 0; k < 9; k++) dsum += creal(At[k] * conj(At[k]));
        }
        double d = 2.0 / ((NC * NC - 1.0) * (ND - 1.0) * V) * dsum;
        if (Dp) Dp[dir] = d;
        avg += d / 4.0;
    }
    return avg;
}
