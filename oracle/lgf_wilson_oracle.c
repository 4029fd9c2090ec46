/*
 * lgf_wilson_oracle.c -- plain FP64 CPU reference for generating SU(3) gauge
 * fields with the Wilson plaquette action S = beta sum_P (1 - Re Tr U_P / 3),
 * the kind of configuration the paper gauge-fixes (its comparison runs use
 * Wilson-action configurations at three couplings).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA generator is checked
 * against.  It shares no code with the CUDA path.
 *
 * Update of one link U = U_mu(x) with staple sum A = sum_{nu != mu}
 *   [U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)]
 * (local weight exp((beta/3) Re Tr(U A))), by SU(2) subgroups (0,1), (0,2),
 * (1,2) in turn (Cabibbo-Marinari): with W = U A and its 2x2 block w on the
 * subgroup, r = (w00 + conj(w11))/2, s = (w01 - conj(w10))/2, k = sqrt(|r|^2 +
 * |s|^2), V = [[r, s], [-conj(s), conj(r)]]/k:
 *   heat bath:       Y ~ sqrt(1 - y0^2) exp(b y0) dy0 (uniform direction),
 *                    b = 2 beta k / 3; R = Y V^dag.  y0 by Kennedy-Pendleton
 *                    rejection for b >= 1.6, else by Creutz's method (proposal
 *                    density exp(b y0) by inverse CDF, accepted with probability
 *                    sqrt(1 - y0^2)); 1.6 is where their acceptance rates cross
 *   overrelaxation:  R = (V^dag)^2 (Re Tr(R W) unchanged)
 * and U <- R U with R embedded in the subgroup.  After the three subgroups,
 * rows 0,1 are Gram-Schmidt orthonormalised and row 2 rebuilt.  A sweep updates
 * direction mu = 0..3, each in two checkerboard halves (even sites, then odd),
 * sites in index order.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 * (link index mu V + s, sweep, 1024 subgroup + draw, 0), uniforms
 * u = (word + 0.5) 2^-32.  Attempt a (< 512) of subgroup g draws counter
 * 1024 g + 2a for y0 (Kennedy-Pendleton: r1..r4; Creutz: u1 for the proposal,
 * u2 for the acceptance) and, once accepted, 1024 g + 2a + 1 for the direction
 * (cos theta = 2 v1 - 1, phi = 2 pi v2).  A subgroup whose 512 attempts all
 * fail is left unchanged (R = 1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef double complex cplx;

static long vol(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long s, int c[4])
{
    for (int mu = 0; mu < 4; mu++) {
        c[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

static long site_of(const int L[4], const int c[4])
{
    long s = 0;
    for (int mu = 3; mu >= 0; mu--) s = s * L[mu] + c[mu];
    return s;
}

static long hop(const int L[4], long s, int mu, int d)
{
    int c[4];
    coords(L, s, c);
    c[mu] = (c[mu] + d + L[mu]) % L[mu];
    return site_of(L, c);
}

/* ---------------------------------------------------------------- Philox4x32-10 */

static void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

static void uniforms(uint64_t seed, uint32_t link, uint32_t sweep, uint32_t draw, double u[4])
{
    uint32_t c[4] = {link, sweep, draw, 0u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    for (int i = 0; i < 4; i++) u[i] = ((double)c[i] + 0.5) * 2.3283064365386962890625e-10;
}

/* the bare generator: out = Philox4x32-10(counter ctr, key) */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    philox(c, key[0], key[1]);
    memcpy(out, c, sizeof c);
}

/* ---------------------------------------------------------------- SU(2) sampler */

/* y0 with density sqrt(1 - y0^2) exp(b y0) on [-1, 1] and a uniform direction:
 * y = (y0, y1, y2, y3), Y = y0 + i (y1 s1 + y2 s2 + y3 s3).  Returns 0 after
 * 512 failed attempts (then y = identity). */
static int su2_sample(double b, uint64_t seed, uint32_t link, uint32_t sweep, int sub, double y[4])
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int a = 0; a < 512; a++) {
        double u[4];
        uniforms(seed, link, sweep, (uint32_t)(1024 * sub + 2 * a), u);
        double y0;
        int ok;
        if (b >= 1.6) {
            /* Kennedy-Pendleton: lambda^2 = (Exp(1) + half a squared normal) / 2b, x0 = 1 - 2 lambda^2 */
            const double c = cos(two_pi * u[1]);
            const double lam2 = -(log(u[0]) + c * c * log(u[2])) / (2.0 * b);
            ok = u[3] * u[3] <= 1.0 - lam2;
            y0 = 1.0 - 2.0 * lam2;
        } else {
            /* Creutz: y0 from exp(b y0) on [-1, 1], accepted with probability sqrt(1 - y0^2) */
            y0 = b > 0 ? 1.0 + log1p((1.0 - u[0]) * expm1(-2.0 * b)) / b : 2.0 * u[0] - 1.0;
            ok = u[1] * u[1] <= 1.0 - y0 * y0;
        }
        if (ok) {
            double v[4];
            uniforms(seed, link, sweep, (uint32_t)(1024 * sub + 2 * a + 1), v);
            const double ct = 2.0 * v[0] - 1.0;
            const double st = sqrt(1.0 - ct * ct);
            const double ph = two_pi * v[1];
            const double rr = sqrt(fmax(1.0 - y0 * y0, 0.0));
            y[0] = y0;
            y[1] = rr * st * cos(ph);
            y[2] = rr * st * sin(ph);
            y[3] = rr * ct;
            return 1;
        }
    }
    y[0] = 1.0;
    y[1] = y[2] = y[3] = 0.0;
    return 0;
}

/* n samples (y0, y1, y2, y3) for one b, links 0..n-1 of sweep 0, subgroup 0 */
void orc_su2_samples(double b, uint64_t seed, int n, double* y)
{
    for (int i = 0; i < n; i++) su2_sample(b, seed, (uint32_t)i, 0u, 0, y + 4 * i);
}

/* ---------------------------------------------------------------- 3x3 helpers */

static void mul(const cplx* a, const cplx* b, cplx* c)
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(c, t, sizeof t);
}

static void dagger(const cplx* a, cplx* b)
{
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) t[3 * i + j] = conj(a[3 * j + i]);
    memcpy(b, t, sizeof t);
}

static void reunit_rows(cplx* m)
{
    double n = 0;
    for (int j = 0; j < 3; j++) n += creal(m[j] * conj(m[j]));
    n = 1.0 / sqrt(n);
    for (int j = 0; j < 3; j++) m[j] *= n;
    cplx ip = 0;
    for (int j = 0; j < 3; j++) ip += conj(m[j]) * m[3 + j];
    double n1 = 0;
    for (int j = 0; j < 3; j++) {
        m[3 + j] -= ip * m[j];
        n1 += creal(m[3 + j] * conj(m[3 + j]));
    }
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; j++) m[3 + j] *= n1;
    m[6] = conj(m[1] * m[5] - m[2] * m[4]);
    m[7] = conj(m[2] * m[3] - m[0] * m[5]);
    m[8] = conj(m[0] * m[4] - m[1] * m[3]);
}

static void staple(const int L[4], const cplx* U, long s, int mu, cplx* A)
{
    const long V = vol(L);
    memset(A, 0, 9 * sizeof(cplx));
    const long sp = hop(L, s, mu, +1);
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        cplx t[9], u[9];
        /* U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
        dagger(U + ((long)mu * V + hop(L, s, nu, +1)) * 9, u);
        mul(U + ((long)nu * V + sp) * 9, u, t);
        dagger(U + ((long)nu * V + s) * 9, u);
        mul(t, u, t);
        for (int e = 0; e < 9; e++) A[e] += t[e];
        /* U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) */
        const long sm = hop(L, s, nu, -1);
        cplx a[9], b[9];
        dagger(U + ((long)nu * V + hop(L, sp, nu, -1)) * 9, a);
        dagger(U + ((long)mu * V + sm) * 9, b);
        mul(a, b, t);
        mul(t, U + ((long)nu * V + sm) * 9, t);
        for (int e = 0; e < 9; e++) A[e] += t[e];
    }
}

/* One link: three SU(2) subgroups, heat bath (mode 0) or overrelaxation (1). */
static void update_link(const int L[4], cplx* U, long s, int mu, double beta, uint64_t seed, uint32_t sweep,
                        int mode)
{
    const long V = vol(L);
    cplx* u = U + ((long)mu * V + s) * 9;
    cplx A[9], W[9];
    staple(L, U, s, mu, A);
    mul(u, A, W);
    static const int sg[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int g = 0; g < 3; g++) {
        const int i = sg[g][0], j = sg[g][1];
        const cplx r = 0.5 * (W[3 * i + i] + conj(W[3 * j + j]));
        const cplx sv = 0.5 * (W[3 * i + j] - conj(W[3 * j + i]));
        const double k = sqrt(creal(r * conj(r)) + creal(sv * conj(sv)));
        if (!(k > 0)) continue;
        /* V = [[a, b], [-conj(b), conj(a)]] with a = r/k, b = s/k */
        const cplx a = r / k, b = sv / k;
        cplx R00, R01, R10, R11;
        if (mode == 0) {
            double y[4];
            su2_sample(2.0 * beta * k / 3.0, seed, (uint32_t)((long)mu * V + s), sweep, g, y);
            /* Y = [[y0 + i y3, y2 + i y1], [-y2 + i y1, y0 - i y3]] ; R = Y V^dag */
            const cplx Y00 = y[0] + I * y[3], Y01 = y[2] + I * y[1];
            const cplx Y10 = -y[2] + I * y[1], Y11 = y[0] - I * y[3];
            /* V^dag = [[conj(a), -b], [conj(b), a]] */
            R00 = Y00 * conj(a) + Y01 * conj(b);
            R01 = -Y00 * b + Y01 * a;
            R10 = Y10 * conj(a) + Y11 * conj(b);
            R11 = -Y10 * b + Y11 * a;
        } else {
            /* R = (V^dag)^2 */
            const cplx D00 = conj(a), D01 = -b, D10 = conj(b), D11 = a;
            R00 = D00 * D00 + D01 * D10;
            R01 = D00 * D01 + D01 * D11;
            R10 = D10 * D00 + D11 * D10;
            R11 = D10 * D01 + D11 * D11;
        }
        /* rows i, j of u and of W: new = R (rows i, j) */
        for (int c = 0; c < 3; c++) {
            const cplx ui = u[3 * i + c], uj = u[3 * j + c];
            u[3 * i + c] = R00 * ui + R01 * uj;
            u[3 * j + c] = R10 * ui + R11 * uj;
            const cplx wi = W[3 * i + c], wj = W[3 * j + c];
            W[3 * i + c] = R00 * wi + R01 * wj;
            W[3 * j + c] = R10 * wi + R11 * wj;
        }
    }
    reunit_rows(u);
}

/* One link update on its own (mode as above), as it would run inside a sweep
 * on the field U: the new U_mu(s) goes to out (3x3), U is left as it was. */
void orc_wilson_link(const int L[4], cplx* U, long s, int mu, double beta, uint64_t seed, uint32_t sweep, int mode,
                     cplx* out)
{
    cplx* u = U + ((long)mu * vol(L) + s) * 9;
    cplx keep[9];
    memcpy(keep, u, sizeof keep);
    update_link(L, U, s, mu, beta, seed, sweep, mode);
    memcpy(out, u, sizeof keep);
    memcpy(u, keep, sizeof keep);
}

/* One sweep over all links: mu = 0..3, even sites then odd sites. */
void orc_wilson_sweep(const int L[4], cplx* U, double beta, uint64_t seed, uint32_t sweep, int mode)
{
    const long V = vol(L);
    for (int mu = 0; mu < 4; mu++)
        for (int par = 0; par < 2; par++)
            for (long s = 0; s < V; s++) {
                int c[4];
                coords(L, s, c);
                if (((c[0] + c[1] + c[2] + c[3]) & 1) != par) continue;
                update_link(L, U, s, mu, beta, seed, sweep, mode);
            }
}

/* Wilson action density: mean over plaquettes of Re Tr U_P / 3 */
double orc_wilson_plaquette(const int L[4], const cplx* U)
{
    const long V = vol(L);
    double acc = 0;
    for (long s = 0; s < V; s++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                cplx a[9], b[9], t[9];
                mul(U + ((long)mu * V + s) * 9, U + ((long)nu * V + hop(L, s, mu, 1)) * 9, t);
                dagger(U + ((long)mu * V + hop(L, s, nu, 1)) * 9, a);
                mul(t, a, t);
                dagger(U + ((long)nu * V + s) * 9, b);
                mul(t, b, t);
                acc += creal(t[0] + t[4] + t[8]) / 3.0;
            }
    return acc / (6.0 * V);
}
