// Reverse-mode derivative (vector-Jacobian product) of one Fourier-accelerated
// steepest-descent step and of the gluon propagator at the smallest momenta,
// FP64.  Gradients of a real loss L follow the convention G_z = dL/dRe z +
// i dL/dIm z, so a first-order change is dL = Re sum conj(G_z) dz, and for
// y = a b:  G_a += G_y conj(b),  G_b += conj(a) G_y;  for Y = A B (matrices):
// G_A += G_Y B^dag, G_B += A^dag G_Y.
//
// The step S: U -> U' with (rows 0,1 stored, row 2 rebuilt as conj(r0 x r1))
//   M(x) = sum_mu [U_mu(x-mu) - U_mu(x)],  Delta = T(M - M^dag),  T(Y) = Y - tr(Y)/3
//   Dt = FA(Delta) (entrywise, real even multiplier: self-adjoint)
//   X = 1 + (alpha/2) Dt,  g = reunit(X) (row Gram-Schmidt, row 2 = conj(r0 x r1))
//   U'_mu(x) = rows 0,1 of g(x) U_mu(x) g^dag(x+mu)
// Backward, given G' (cotangent of the full output U', row 2 included):
//   b1 (per link): G01 = G'_rows01 + (row-2 rebuild)^T G'_row2;
//                  G_U^direct = g^dag P^T G01 g(x+mu);  G_g(x) rows 0,1 += G01 g(x+mu) U^dag;
//                  Q = G01^dag P g(x) U  (the part of G_g(x+mu))
//   b2 (per site): G_g(y) = self + sum_mu Q_mu(y-mu); Gram-Schmidt backward -> G_X;
//                  G_Dt rows 0,1 = (alpha/2) G_X   (six complex fields)
//   FA on the six fields
//   b4 (per site): G_M = T(G_Delta) - T(G_Delta)^dag;
//                  G_U_mu(x) = G_U^direct + G_M(x+mu) - G_M(x); (row-2 rebuild)^T -> rows 0,1
#pragma once
#include "lgf_kernels.cuh"

namespace lgf {

using C = cx<double>;

__device__ __forceinline__ C cneg(C a) { return mk<double>(-a.re, -a.im); }
__device__ __forceinline__ C cscale(C a, double s) { return mk<double>(a.re * s, a.im * s); }
// i * a / 2
__device__ __forceinline__ C ihalf(C a) { return mk<double>(-0.5 * a.im, 0.5 * a.re); }

// Accumulate into G_r0, G_r1 the pull-back of G_r2 through r2 = conj(r0 x r1).
__device__ __forceinline__ void row2_bwd(const C* r0, const C* r1, const C* g2, C* G0, C* G1)
{
    // entry 0: conj(r0_1 r1_2 - r0_2 r1_1)
    G0[1] = G0[1] + conjg(cmul(g2[0], r1[2]));
    G1[2] = G1[2] + conjg(cmul(g2[0], r0[1]));
    G0[2] = G0[2] - conjg(cmul(g2[0], r1[1]));
    G1[1] = G1[1] - conjg(cmul(g2[0], r0[2]));
    // entry 1: conj(r0_2 r1_0 - r0_0 r1_2)
    G0[2] = G0[2] + conjg(cmul(g2[1], r1[0]));
    G1[0] = G1[0] + conjg(cmul(g2[1], r0[2]));
    G0[0] = G0[0] - conjg(cmul(g2[1], r1[2]));
    G1[2] = G1[2] - conjg(cmul(g2[1], r0[0]));
    // entry 2: conj(r0_0 r1_1 - r0_1 r1_0)
    G0[0] = G0[0] + conjg(cmul(g2[2], r1[1]));
    G1[1] = G1[1] + conjg(cmul(g2[2], r0[0]));
    G0[1] = G0[1] - conjg(cmul(g2[2], r1[0]));
    G1[0] = G1[0] - conjg(cmul(g2[2], r0[1]));
}

// pull-back through r = x / |x| (three complex components)
__device__ __forceinline__ void normalize_bwd(const C* r, double n, const C* Gr, C* Gx)
{
    double s = 0;
#pragma unroll
    for (int j = 0; j < 3; j++) s += r[j].re * Gr[j].re + r[j].im * Gr[j].im;  // Re <r, Gr>
#pragma unroll
    for (int j = 0; j < 3; j++) Gx[j] = cscale(Gr[j] - cscale(r[j], s), 1.0 / n);
}

template <typename P> __device__ __forceinline__ void load9(const P* __restrict__ p, int V, int s, C* m)
{
#pragma unroll
    for (int e = 0; e < 9; e++) m[e] = ld<double>(p + (size_t)e * V + s);
}
__device__ __forceinline__ void store9(double2* __restrict__ p, int V, int s, const C* m)
{
#pragma unroll
    for (int e = 0; e < 9; e++) st<double>(p + (size_t)e * V + s, m[e]);
}

// ---------------------------------------------------------------- forward pieces

// g(x) = reunit(1 + alpha/2 Dt(x)) from the four packed spatial fields of Dt
static __global__ void k_g_from_dt(int V, const double2* __restrict__ Fd, double2* __restrict__ g, double alpha)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const double h = 0.5 * alpha;
    const double2 f0 = Fd[s], f1 = Fd[(size_t)V + s], f2 = Fd[(size_t)2 * V + s], f3 = Fd[(size_t)3 * V + s];
    C X[6];
    X[0] = mk<double>(1.0, h * f3.x);
    X[1] = mk<double>(h * f0.x, h * f0.y);
    X[2] = mk<double>(h * f1.x, h * f1.y);
    X[3] = mk<double>(-h * f0.x, h * f0.y);
    X[4] = mk<double>(1.0, h * f3.y);
    X[5] = mk<double>(h * f2.x, h * f2.y);
    C gm[9];
    reunit_rows(X, gm);
    store9(g, V, s, gm);
}

// [4][V][3][3] interleaved complex128 -> [4][9][V] planes (full matrices)
static __global__ void k_pack_full(int V, const double* __restrict__ in, double2* __restrict__ out)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4L * V) return;
    const int mu = (int)(idx / V), s = (int)(idx - (long)mu * V);
    const double* p = in + idx * 18;
#pragma unroll
    for (int e = 0; e < 9; e++) out[(size_t)(mu * 9 + e) * V + s] = make_double2(p[2 * e], p[2 * e + 1]);
}

// [4][9][V] planes -> [4][V][3][3] interleaved complex128
static __global__ void k_unpack_planes(int V, const double2* __restrict__ in, double* __restrict__ out)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4L * V) return;
    const int mu = (int)(idx / V), s = (int)(idx - (long)mu * V);
    double* p = out + idx * 18;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        const double2 v = in[(size_t)(mu * 9 + e) * V + s];
        p[2 * e] = v.x;
        p[2 * e + 1] = v.y;
    }
}

// ---------------------------------------------------------------- step backward

// b1: one thread per site, its four links.  Gp: cotangent of U' ([4][9][V]).
static __global__ void __launch_bounds__(128) k_bwd_update(Lat d, const double2* __restrict__ U,
                                                           const double2* __restrict__ g,
                                                           const double2* __restrict__ Gp, double2* __restrict__ Gud,
                                                           double2* __restrict__ Ggs, double2* __restrict__ Q)
{
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    C gx[9];
    load9(g, V, s, gx);
    C Gg[6];
#pragma unroll
    for (int e = 0; e < 6; e++) Gg[e] = mk<double>(0, 0);
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
        C u[9];
        load_link<double>(U, V, d.ne, mu, s, u);
        C gn[9];
        load9(g, V, site_shift(d, s, c[mu], mu, +1), gn);
        // Vr = rows 0,1 of g(x) U; Up = Vr gn^dag
        C Vr[6], Up[6];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C acc = cmul(gx[3 * i], u[j]);
                acc = cmac(acc, gx[3 * i + 1], u[3 + j]);
                acc = cmac(acc, gx[3 * i + 2], u[6 + j]);
                Vr[3 * i + j] = acc;
            }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C acc = cmulc(Vr[3 * i], gn[3 * j]);
                acc = cmacc(acc, Vr[3 * i + 1], gn[3 * j + 1]);
                acc = cmacc(acc, Vr[3 * i + 2], gn[3 * j + 2]);
                Up[3 * i + j] = acc;
            }
        // G01 = rows 0,1 of the cotangent + pull-back of its row 2 through the rebuild
        C G01[6], g2[3];
#pragma unroll
        for (int e = 0; e < 6; e++) G01[e] = ld<double>(Gp + (size_t)(mu * 9 + e) * V + s);
#pragma unroll
        for (int e = 0; e < 3; e++) g2[e] = ld<double>(Gp + (size_t)(mu * 9 + 6 + e) * V + s);
        row2_bwd(Up, Up + 3, g2, G01, G01 + 3);
        // Y = G01 gn (2x3)
        C Y[6];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C acc = cmul(G01[3 * i], gn[j]);
                acc = cmac(acc, G01[3 * i + 1], gn[3 + j]);
                acc = cmac(acc, G01[3 * i + 2], gn[6 + j]);
                Y[3 * i + j] = acc;
            }
        // G_U^direct = (rows 0,1 of g)^dag Y (3x3)
        C Gd[9];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                C acc = cmul(conjg(gx[a]), Y[b]);
                acc = cmac(acc, conjg(gx[3 + a]), Y[3 + b]);
                Gd[3 * a + b] = acc;
            }
        store9(Gud + (size_t)mu * 9 * V, V, s, Gd);
        // G_g(x) rows 0,1 += Y U^dag
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C acc = cmacc(Gg[3 * i + j], Y[3 * i], u[3 * j]);
                acc = cmacc(acc, Y[3 * i + 1], u[3 * j + 1]);
                Gg[3 * i + j] = cmacc(acc, Y[3 * i + 2], u[3 * j + 2]);
            }
        // Q = G01^dag Vr (3x3): the contribution to G_g(x+mu)
        C Qm[9];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                C acc = cmul(conjg(G01[a]), Vr[b]);
                acc = cmac(acc, conjg(G01[3 + a]), Vr[3 + b]);
                Qm[3 * a + b] = acc;
            }
        store9(Q + (size_t)mu * 9 * V, V, s, Qm);
    }
#pragma unroll
    for (int e = 0; e < 6; e++) st<double>(Ggs + (size_t)e * V + s, Gg[e]);
}

// b2: one thread per site.  G_g -> Gram-Schmidt backward -> G_Dt rows 0,1,
// written as six fields into FA (fields 00,01,02,10) and FB (11,12,0,0).
static __global__ void k_bwd_reunit(Lat d, const double2* __restrict__ Fdt, const double2* __restrict__ Ggs,
                                    const double2* __restrict__ Q, double alpha, double2* __restrict__ FA,
                                    double2* __restrict__ FB)
{
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    C Gg[9];
#pragma unroll
    for (int e = 0; e < 6; e++) Gg[e] = ld<double>(Ggs + (size_t)e * V + s);
#pragma unroll
    for (int e = 6; e < 9; e++) Gg[e] = mk<double>(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int sb = site_shift(d, s, c[mu], mu, -1);
#pragma unroll
        for (int e = 0; e < 9; e++) Gg[e] = Gg[e] + ld<double>(Q + (size_t)(mu * 9 + e) * V + sb);
    }
    // recompute the Gram-Schmidt forward from X = 1 + h Dt
    const double h = 0.5 * alpha;
    const double2 f0 = Fdt[s], f1 = Fdt[(size_t)V + s], f2 = Fdt[(size_t)2 * V + s], f3 = Fdt[(size_t)3 * V + s];
    C X[6];
    X[0] = mk<double>(1.0, h * f3.x);
    X[1] = mk<double>(h * f0.x, h * f0.y);
    X[2] = mk<double>(h * f1.x, h * f1.y);
    X[3] = mk<double>(-h * f0.x, h * f0.y);
    X[4] = mk<double>(1.0, h * f3.y);
    X[5] = mk<double>(h * f2.x, h * f2.y);
    const double n0 = sqrt(norm2(X[0]) + norm2(X[1]) + norm2(X[2]));
    C r0[3], r1[3], v[3];
#pragma unroll
    for (int j = 0; j < 3; j++) r0[j] = cscale(X[j], 1.0 / n0);
    C ip = cmulc(X[3], r0[0]);
    ip = cmacc(ip, X[4], r0[1]);
    ip = cmacc(ip, X[5], r0[2]);
#pragma unroll
    for (int j = 0; j < 3; j++) v[j] = X[3 + j] - cmul(ip, r0[j]);
    const double n1 = sqrt(norm2(v[0]) + norm2(v[1]) + norm2(v[2]));
#pragma unroll
    for (int j = 0; j < 3; j++) r1[j] = cscale(v[j], 1.0 / n1);
    // backward
    C G0[3] = {Gg[0], Gg[1], Gg[2]}, G1[3] = {Gg[3], Gg[4], Gg[5]};
    row2_bwd(r0, r1, Gg + 6, G0, G1);
    C Gv[3], GX0[3], GX1[3];
    normalize_bwd(r1, n1, G1, Gv);
    C Gip = mk<double>(0, 0);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        GX1[j] = Gv[j];
        Gip = Gip - cmulc(Gv[j], r0[j]);           // v = X1 - ip r0
        G0[j] = G0[j] - cmul(conjg(ip), Gv[j]);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        G0[j] = G0[j] + cmul(conjg(Gip), X[3 + j]);  // ip = sum conj(r0_j) X1_j
        GX1[j] = GX1[j] + cmul(r0[j], Gip);
    }
    normalize_bwd(r0, n0, G0, GX0);
    FA[s] = make_double2(h * GX0[0].re, h * GX0[0].im);
    FA[(size_t)V + s] = make_double2(h * GX0[1].re, h * GX0[1].im);
    FA[(size_t)2 * V + s] = make_double2(h * GX0[2].re, h * GX0[2].im);
    FA[(size_t)3 * V + s] = make_double2(h * GX1[0].re, h * GX1[0].im);
    FB[s] = make_double2(h * GX1[1].re, h * GX1[1].im);
    FB[(size_t)V + s] = make_double2(h * GX1[2].re, h * GX1[2].im);
    FB[(size_t)2 * V + s] = make_double2(0.0, 0.0);
    FB[(size_t)3 * V + s] = make_double2(0.0, 0.0);
}

// G_M at site s from G_Delta rows 0,1 (row 2 of G_Delta is zero)
__device__ __forceinline__ void grad_M(const double2* __restrict__ FA, const double2* __restrict__ FB, int V, int s,
                                       C* GM)
{
    C Gd[9];
    Gd[0] = ld<double>(FA + s);
    Gd[1] = ld<double>(FA + (size_t)V + s);
    Gd[2] = ld<double>(FA + (size_t)2 * V + s);
    Gd[3] = ld<double>(FA + (size_t)3 * V + s);
    Gd[4] = ld<double>(FB + s);
    Gd[5] = ld<double>(FB + (size_t)V + s);
    Gd[6] = Gd[7] = Gd[8] = mk<double>(0, 0);
    const C t = cscale(Gd[0] + Gd[4], 1.0 / 3.0);
    Gd[0] = Gd[0] - t;
    Gd[4] = Gd[4] - t;
    Gd[8] = Gd[8] - t;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) GM[3 * i + j] = Gd[3 * i + j] - conjg(Gd[3 * j + i]);
}

// b4: one thread per site; output cotangent of the input links (rows 0,1; row 2 zero)
static __global__ void k_bwd_delta(Lat d, const double2* __restrict__ U, const double2* __restrict__ FA,
                                   const double2* __restrict__ FB, const double2* __restrict__ Gud,
                                   double2* __restrict__ Gin)
{
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    C GMx[9];
    grad_M(FA, FB, V, s, GMx);
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
        C GMn[9], Gu[9];
        grad_M(FA, FB, V, site_shift(d, s, c[mu], mu, +1), GMn);
        load9(Gud + (size_t)mu * 9 * V, V, s, Gu);
#pragma unroll
        for (int e = 0; e < 9; e++) Gu[e] = Gu[e] + GMn[e] - GMx[e];
        C u[9];
        load_link<double>(U, V, d.ne, mu, s, u);
        row2_bwd(u, u + 3, Gu + 6, Gu, Gu + 3);
        Gu[6] = Gu[7] = Gu[8] = mk<double>(0, 0);
        store9(Gin + (size_t)mu * 9 * V, V, s, Gu);
    }
}

// ---------------------------------------------------------------- gluon propagator

// Partial sums of A~_mu(p_nu) = sum_x exp(-2 pi i x_nu / L_nu) A_mu(x) over the
// block's sites; grid.y = 4 nu + mu.  A = (U - U^dag)/(2i) - tr/3 (9 entries).
static __global__ void __launch_bounds__(256) k_gluon_partial(Lat d, const double2* __restrict__ U,
                                                              const double2* __restrict__ tw0,
                                                              const double2* __restrict__ tw1,
                                                              const double2* __restrict__ tw2,
                                                              const double2* __restrict__ tw3,
                                                              double2* __restrict__ part /* [16][nbx][9] */)
{
    __shared__ double red[2][9][8];
    const int V = d.V;
    const int nu = blockIdx.y >> 2, mu = blockIdx.y & 3;
    const double2* tw = nu == 0 ? tw0 : nu == 1 ? tw1 : nu == 2 ? tw2 : tw3;
    C acc[9];
#pragma unroll
    for (int e = 0; e < 9; e++) acc[e] = mk<double>(0, 0);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
        int c[4];
        site_coords(d, s, c);
        C u[9];
        load_link<double>(U, V, d.ne, mu, s, u);
        C A[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const C y = u[3 * i + j] - conjg(u[3 * j + i]);  // (U - U^dag)_ij; / (2i) = -i/2
                A[3 * i + j] = mk<double>(0.5 * y.im, -0.5 * y.re);
            }
        const C t = cscale(A[0] + A[4] + A[8], 1.0 / 3.0);
        A[0] = A[0] - t;
        A[4] = A[4] - t;
        A[8] = A[8] - t;
        const C w = ld<double>(tw + c[nu]);  // exp(-2 pi i x_nu / L_nu)
#pragma unroll
        for (int e = 0; e < 9; e++) acc[e] = cmac(acc[e], w, A[e]);
    }
    // block reduction in a fixed order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < 9; e++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc[e].re += __shfl_down_sync(0xffffffffu, acc[e].re, o);
            acc[e].im += __shfl_down_sync(0xffffffffu, acc[e].im, o);
        }
        if (lane == 0) {
            red[0][e][wid] = acc[e].re;
            red[1][e][wid] = acc[e].im;
        }
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        const int e = threadIdx.x;
        double re = 0, im = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            re += red[0][e][w];
            im += red[1][e][w];
        }
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 9 + e] = make_double2(re, im);
    }
}

// One block of 144 threads: At[16][9] = sums of the partials (block order),
// then D_nu = c sum_mu sum_e |At|^2 (c = 2 / ((N_c^2-1)(N_d-1) V)) for the four
// momenta and their mean: D[0..3], D[4].
static __global__ void k_gluon_final(int nbx, double c, const double2* __restrict__ part, double2* __restrict__ At,
                                     double* __restrict__ D)
{
    __shared__ double sq[144];
    const int k = threadIdx.x;  // (nu mu) * 9 + e
    if (k < 144) {
        const int nm = k / 9, e = k - nm * 9;
        double re = 0, im = 0;
        for (int b = 0; b < nbx; b++) {
            const double2 v = part[((size_t)nm * nbx + b) * 9 + e];
            re += v.x;
            im += v.y;
        }
        At[k] = make_double2(re, im);
        sq[k] = re * re + im * im;
    }
    __syncthreads();
    if (k == 0) {
        double avg = 0;
        for (int nu = 0; nu < 4; nu++) {
            double t = 0;
            for (int j = 0; j < 36; j++) t += sq[nu * 36 + j];
            D[nu] = c * t;
            avg += 0.25 * c * t;
        }
        D[4] = avg;
    }
}

// G_U from dL/dD: G_A_mu(x) = sum_nu (gD c / 4) 2 A~_{nu mu} exp(+2 pi i x_nu / L_nu),
// G_U = (i/2)(T(G_A) + T(G_A)^dag), then the row-2 pull-back.  Writes [4][9][V].
static __global__ void k_gluon_bwd(Lat d, const double2* __restrict__ U, const double2* __restrict__ At, double coef,
                                   const double2* __restrict__ tw0, const double2* __restrict__ tw1,
                                   const double2* __restrict__ tw2, const double2* __restrict__ tw3,
                                   double2* __restrict__ Gout)
{
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    const double2* tws[4] = {tw0, tw1, tw2, tw3};
    C w[4];
#pragma unroll
    for (int nu = 0; nu < 4; nu++) w[nu] = conjg(ld<double>(tws[nu] + c[nu]));  // exp(+2 pi i x_nu/L_nu)
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
        C GA[9];
#pragma unroll
        for (int e = 0; e < 9; e++) {
            C a = mk<double>(0, 0);
#pragma unroll
            for (int nu = 0; nu < 4; nu++) a = cmac(a, w[nu], ld<double>(At + (nu * 4 + mu) * 9 + e));
            GA[e] = cscale(a, coef);
        }
        const C t = cscale(GA[0] + GA[4] + GA[8], 1.0 / 3.0);
        GA[0] = GA[0] - t;
        GA[4] = GA[4] - t;
        GA[8] = GA[8] - t;
        C Gu[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Gu[3 * i + j] = ihalf(GA[3 * i + j] + conjg(GA[3 * j + i]));
        C u[9];
        load_link<double>(U, V, d.ne, mu, s, u);
        row2_bwd(u, u + 3, Gu + 6, Gu, Gu + 3);
        Gu[6] = Gu[7] = Gu[8] = mk<double>(0, 0);
        store9(Gout + (size_t)mu * 9 * V, V, s, Gu);
    }
}

}  // namespace lgf
