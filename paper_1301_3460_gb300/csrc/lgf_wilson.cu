// Wilson-action Monte Carlo of the links a context holds: SU(3) configurations
// of the kind the paper's 32^4 comparison runs gauge-fix (Wilson action at three
// couplings), generated on the device so that they go straight into the fixing
// loop.  The paper does not describe its generator; this one is the standard
// Cabibbo-Marinari heat bath with overrelaxation.
//
// Action S = beta sum_P (1 - Re Tr U_P / 3).  The links U_mu(x) with x of one
// checkerboard parity share no plaquette, so one launch updates all of them at
// once: one thread per site of that parity, direction mu fixed per launch.  Per
// link, with the staple sum
//   A = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//                    + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu),
// W = U A and the SU(2) subgroups (0,1), (0,2), (1,2) in turn: the 2x2 block w
// of W gives r = (w_ii + conj w_jj)/2, s = (w_ij - conj w_ji)/2, k = |(r, s)|
// and the SU(2) element V = [[r, s], [-conj s, conj r]]/k, and the link becomes
// R U with R in the subgroup:
//   heat bath      R = Y V^dag, Y ~ sqrt(1 - y0^2) exp(b y0), b = 2 beta k / 3,
//                  uniform direction (Kennedy-Pendleton for b >= 1.6, Creutz
//                  below, where their acceptance rates cross)
//   overrelaxation R = (V^dag)^2 (leaves Re Tr(U A) unchanged)
// then rows 0,1 are Gram-Schmidt orthonormalised and row 2 rebuilt.
//
// Random numbers are counter-based (Philox4x32-10, Salmon et al., SC'11): key =
// the 64-bit seed, counter (mu V + s, sweep, 1024 subgroup + draw, 0), so a
// result depends on neither the launch shape nor the thread order.  Attempt a of
// subgroup g reads draw 2a (y0) and, once accepted, 2a + 1 (direction); after
// 512 failed attempts the subgroup is left unchanged.
//
// Every step is FP64.  Per link: 12 3x3 complex products for the staples (the
// six of two SU(3) links with row 2 rebuilt instead of multiplied out), one for
// W, the sampler's transcendental functions; the kernel is bound by the FP64
// pipe.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lgf_common.cuh"
#include "lgf_launch.h"

namespace lgf {
namespace {

using C = cx<double>;

constexpr int kWilsonThreads = 128;
constexpr int kPlaqThreads = 256;
constexpr int kPlaqBlocks = 1216;  // 8 per SM on 152 SMs; grid-stride beyond

// matrix helpers for T = double (the FP64 generator) and T = float (the staples
// of the FP32 one); links are FP64 in memory in both cases

template <typename T> __device__ __forceinline__ cx<T> ldl(const double2* p)
{
    const double2 v = __ldg(p);
    return mk<T>((T)v.x, (T)v.y);
}
template <typename T> __device__ __forceinline__ cx<T> ldl(const float2* p)
{
    const float2 v = __ldg(p);
    return mk<T>((T)v.x, (T)v.y);
}

template <typename T, typename S>
__device__ __forceinline__ void load3(const S* __restrict__ U, int V, int ne, int mu, int s, cx<T>* m)
{
#pragma unroll
    for (int e = 0; e < 6; e++) m[e] = ldl<T>(U + (size_t)(mu * ne + e) * V + s);
    if (ne == 9) {
#pragma unroll
        for (int e = 6; e < 9; e++) m[e] = ldl<T>(U + (size_t)(mu * 9 + e) * V + s);
    } else {
        complete_row2(m, m + 6);
    }
}

// rows 0,1 of a link (all that a product whose row 2 is rebuilt needs)
template <typename T, typename S>
__device__ __forceinline__ void load2(const S* __restrict__ U, int V, int ne, int mu, int s, cx<T>* m)
{
#pragma unroll
    for (int e = 0; e < 6; e++) m[e] = ldl<T>(U + (size_t)(mu * ne + e) * V + s);
}

// c = a b for a, b in SU(3): rows 0,1 multiplied out, row 2 = conj(row0 x row1)
// (a's row 2 is not read)
template <typename T> __device__ __forceinline__ void mm_su3(const cx<T>* a, const cx<T>* b, cx<T>* c)
{
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> t = cmul(a[3 * i], b[j]);
            t = cmac(t, a[3 * i + 1], b[3 + j]);
            c[3 * i + j] = cmac(t, a[3 * i + 2], b[6 + j]);
        }
    complete_row2(c, c + 6);
}

// c = a b
template <typename T> __device__ __forceinline__ void mm(const cx<T>* a, const cx<T>* b, cx<T>* c)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> t = cmul(a[3 * i], b[j]);
            t = cmac(t, a[3 * i + 1], b[3 + j]);
            c[3 * i + j] = cmac(t, a[3 * i + 2], b[6 + j]);
        }
}

// acc += a b^dag
template <typename T> __device__ __forceinline__ void mm_nd_acc(const cx<T>* a, const cx<T>* b, cx<T>* acc)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> t = acc[3 * i + j];
#pragma unroll
            for (int k = 0; k < 3; k++) t = cmacc(t, a[3 * i + k], b[3 * j + k]);
            acc[3 * i + j] = t;
        }
}

// acc += a^dag b
template <typename T> __device__ __forceinline__ void mm_dn_acc(const cx<T>* a, const cx<T>* b, cx<T>* acc)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> t = acc[3 * i + j];
#pragma unroll
            for (int k = 0; k < 3; k++) t = cmacc(t, b[3 * k + j], a[3 * k + i]);
            acc[3 * i + j] = t;
        }
}

// staple sum A of link (mu, s) of parity c
template <typename T, typename S>
__device__ __forceinline__ void staple_sum(const Lat& d, const S* __restrict__ U, int mu, int s, const int* c,
                                           cx<T>* A)
{
    const int V = d.V, ne = d.ne;
#pragma unroll
    for (int e = 0; e < 9; e++) A[e] = mk<T>(0, 0);
    const int sp = site_shift(d, s, c[mu], mu, +1);
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const int snp = site_shift(d, s, c[nu], nu, +1);
        const int snm = site_shift(d, s, c[nu], nu, -1);
        const int spm = site_shift(d, sp, c[nu], nu, -1);  // x + mu - nu
        cx<T> a[9], b[9], q[9];
        load2<T>(U, V, ne, nu, s, a);
        load3<T>(U, V, ne, mu, snp, b);
        mm_su3<T>(a, b, q);             // U_nu(x) U_mu(x+nu)
        load3<T>(U, V, ne, nu, sp, a);
        mm_nd_acc<T>(a, q, A);          // + U_nu(x+mu) q^dag
        load2<T>(U, V, ne, mu, snm, a);
        load3<T>(U, V, ne, nu, spm, b);
        mm_su3<T>(a, b, q);             // U_mu(x-nu) U_nu(x+mu-nu)
        load3<T>(U, V, ne, nu, snm, a);
        mm_dn_acc<T>(q, a, A);          // + q^dag U_nu(x-nu)
    }
}

// ---------------------------------------------------------------- Philox4x32-10

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// four uniforms (word + 1/2) 2^-32 in (0, 1), exact in FP64
__device__ __forceinline__ void draw4(uint32_t k0, uint32_t k1, uint32_t link, uint32_t sweep, uint32_t n, double u[4])
{
    uint32_t c[4] = {link, sweep, n, 0u};
    philox(c, k0, k1);
#pragma unroll
    for (int i = 0; i < 4; i++) u[i] = fma((double)c[i], 0x1p-32, 0x1p-33);
}

// y = (y0, y1, y2, y3) with y0 ~ sqrt(1 - y0^2) exp(b y0) on [-1, 1] and the
// direction uniform on the 2-sphere; the identity after 512 failed attempts.
__device__ __noinline__ void su2_draw(double b, uint32_t k0, uint32_t k1, uint32_t link, uint32_t sweep, int sub,
                                      double y[4])
{
    const bool kp = b >= 1.6;
    const double ib = b > 0 ? 1.0 / b : 0.0;
    const double e2b = kp ? 0.0 : expm1(-2.0 * b);
    for (int a = 0; a < 512; a++) {
        double u[4];
        draw4(k0, k1, link, sweep, (uint32_t)(1024 * sub + 2 * a), u);
        double y0;
        bool ok;
        if (kp) {
            // Kennedy-Pendleton: lambda^2 = (an Exp(1) + half a squared normal) / 2b
            const double c = cospi(2.0 * u[1]);
            const double lam2 = -(log(u[0]) + c * c * log(u[2])) * (0.5 * ib);
            ok = u[3] * u[3] <= 1.0 - lam2;
            y0 = 1.0 - 2.0 * lam2;
        } else {
            // Creutz: proposal exp(b y0) by its inverse distribution function
            y0 = b > 0 ? 1.0 + log1p((1.0 - u[0]) * e2b) * ib : 2.0 * u[0] - 1.0;
            ok = u[1] * u[1] <= 1.0 - y0 * y0;
        }
        if (ok) {
            double v[4];
            draw4(k0, k1, link, sweep, (uint32_t)(1024 * sub + 2 * a + 1), v);
            const double ct = 2.0 * v[0] - 1.0;
            const double st = sqrt(1.0 - ct * ct);
            double sp, cp;
            sincospi(2.0 * v[1], &sp, &cp);
            const double rr = sqrt(fmax(1.0 - y0 * y0, 0.0));
            y[0] = y0;
            y[1] = rr * st * cp;
            y[2] = rr * st * sp;
            y[3] = rr * ct;
            return;
        }
    }
    y[0] = 1.0;
    y[1] = y[2] = y[3] = 0.0;
}

// rows i, j of m <- R (rows i, j)
template <int I, int J, typename T>
__device__ __forceinline__ void rot_rows(cx<T>* m, cx<T> R00, cx<T> R01, cx<T> R10, cx<T> R11)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cx<T> mi = m[3 * I + c], mj = m[3 * J + c];
        m[3 * I + c] = cmac(cmul(R00, mi), R01, mj);
        m[3 * J + c] = cmac(cmul(R10, mi), R11, mj);
    }
}

template <int MODE, int I, int J>
__device__ __forceinline__ void subgroup(C* u, C* w, double beta23, uint32_t k0, uint32_t k1, uint32_t link,
                                         uint32_t sweep, int sub)
{
    const C wii = w[3 * I + I], wjj = w[3 * J + J], wij = w[3 * I + J], wji = w[3 * J + I];
    const C r = mk(0.5 * (wii.re + wjj.re), 0.5 * (wii.im - wjj.im));
    const C s = mk(0.5 * (wij.re - wji.re), 0.5 * (wij.im + wji.im));
    const double k2 = r.re * r.re + r.im * r.im + s.re * s.re + s.im * s.im;
    if (!(k2 > 0)) return;
    const double ik = rsqrt(k2);
    const C a = r * ik, b = s * ik;
    C R00, R01, R10, R11;
    if (MODE == 0) {
        double y[4];
        su2_draw(beta23 * (k2 * ik), k0, k1, link, sweep, sub, y);
        // Y = y0 + i (y1 s1 + y2 s2 + y3 s3); R = Y V^dag, V^dag = [[conj a, -b], [conj b, a]]
        const C Y00 = mk(y[0], y[3]), Y01 = mk(y[2], y[1]), Y10 = mk(-y[2], y[1]), Y11 = mk(y[0], -y[3]);
        const C nb = mk(-b.re, -b.im);
        R00 = cmac(cmul(Y00, conjg(a)), Y01, conjg(b));
        R01 = cmac(cmul(Y00, nb), Y01, a);
        R10 = cmac(cmul(Y10, conjg(a)), Y11, conjg(b));
        R11 = cmac(cmul(Y10, nb), Y11, a);
    } else {
        // R = (V^dag)^2
        const C D00 = conjg(a), D01 = mk(-b.re, -b.im), D10 = conjg(b), D11 = a;
        R00 = cmac(cmul(D00, D00), D01, D10);
        R01 = cmac(cmul(D00, D01), D01, D11);
        R10 = cmac(cmul(D10, D00), D11, D10);
        R11 = cmac(cmul(D10, D01), D11, D11);
    }
    rot_rows<I, J>(u, R00, R01, R10, R11);
    rot_rows<I, J>(w, R00, R01, R10, R11);
}

// Gram-Schmidt of rows 0, 1 (row 2 untouched)
__device__ __forceinline__ void orthonormal_rows01(C* m)
{
    double n0 = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) n0 += norm2(m[c]);
    n0 = rsqrt(n0);
#pragma unroll
    for (int c = 0; c < 3; c++) m[c] = m[c] * n0;
    C ip = mk(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 3; c++) ip = cmacc(ip, m[3 + c], m[c]);  // sum conj(row0) row1
    double n1 = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        m[3 + c] = m[3 + c] - cmul(ip, m[c]);
        n1 += norm2(m[3 + c]);
    }
    n1 = rsqrt(n1);
#pragma unroll
    for (int c = 0; c < 3; c++) m[3 + c] = m[3 + c] * n1;
}

// Gram-Schmidt of rows 0, 1 and row 2 = conj(row0 x row1)
__device__ __forceinline__ void reunit(C* m)
{
    orthonormal_rows01(m);
    complete_row2(m, m + 6);
}

template <int MODE>
__global__ void __launch_bounds__(kWilsonThreads) k_wilson(Lat d, double2* __restrict__ U, int mu, int parity,
                                                           double beta, uint32_t k0, uint32_t k1, uint32_t sweep)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= (d.V >> 1)) return;
    // site of the given parity with pair index h = s / 2 (Lx is even)
    const int hx = d.L[0] >> 1;
    int c[4];
    int r = h / hx;
    const int xh = h - r * hx;
    c[1] = r % d.L[1];
    r /= d.L[1];
    c[2] = r % d.L[2];
    c[3] = r / d.L[2];
    c[0] = 2 * xh + ((parity + c[1] + c[2] + c[3]) & 1);
    const int s = c[0] + d.stride[1] * c[1] + d.stride[2] * c[2] + d.stride[3] * c[3];
    const int V = d.V, ne = d.ne;

    C A[9];
    staple_sum<double>(d, U, mu, s, c, A);
    C u[9], w[9];
    load3<double>(U, V, ne, mu, s, u);
    mm<double>(u, A, w);
    const uint32_t link = (uint32_t)mu * (uint32_t)V + (uint32_t)s;
    const double beta23 = beta * (2.0 / 3.0);  // b = 2 beta k / 3
    subgroup<MODE, 0, 1>(u, w, beta23, k0, k1, link, sweep, 0);
    subgroup<MODE, 0, 2>(u, w, beta23, k0, k1, link, sweep, 1);
    subgroup<MODE, 1, 2>(u, w, beta23, k0, k1, link, sweep, 2);
    reunit(u);
#pragma unroll
    for (int e = 0; e < 6; e++) st<double>(U + (size_t)(mu * ne + e) * V + s, u[e]);
    if (ne == 9) {
#pragma unroll
        for (int e = 6; e < 9; e++) st<double>(U + (size_t)(mu * 9 + e) * V + s, u[e]);
    }
}

// ---------------------------------------------------------------- FP32 generator

// The same update with the staples, W, the SU(2) draws and the rotation of the
// link in FP32, all read from the FP32 copy (links stay FP64 in memory: rows 0,1
// of the rotated link are re-orthonormalised in FP64, so the stored link stays in
// SU(3) to FP64 rounding).  A Markov chain of its own:
// the heat bath samples exp((beta/3) Re Tr(U A)) with A known to FP32 rounding,
// and its uniforms take the top 24 bits of the same Philox words.

__device__ __forceinline__ void draw4f(uint32_t k0, uint32_t k1, uint32_t link, uint32_t sweep, uint32_t n, float u[4])
{
    uint32_t c[4] = {link, sweep, n, 0u};
    philox(c, k0, k1);
#pragma unroll
    for (int i = 0; i < 4; i++) u[i] = fmaf((float)(c[i] >> 8), 0x1p-24f, 0x1p-25f);
}

__device__ __noinline__ void su2_draw_f(float b, uint32_t k0, uint32_t k1, uint32_t link, uint32_t sweep, int sub,
                                        float y[4])
{
    const bool kp = b >= 1.6f;
    const float ib = b > 0 ? 1.0f / b : 0.0f;
    const float e2b = kp ? 0.0f : expm1f(-2.0f * b);
    for (int a = 0; a < 512; a++) {
        float u[4];
        draw4f(k0, k1, link, sweep, (uint32_t)(1024 * sub + 2 * a), u);
        float y0;
        bool ok;
        if (kp) {
            const float c = cospif(2.0f * u[1]);
            const float lam2 = -(logf(u[0]) + c * c * logf(u[2])) * (0.5f * ib);
            ok = u[3] * u[3] <= 1.0f - lam2;
            y0 = 1.0f - 2.0f * lam2;
        } else {
            y0 = b > 0 ? 1.0f + log1pf((1.0f - u[0]) * e2b) * ib : 2.0f * u[0] - 1.0f;
            ok = u[1] * u[1] <= 1.0f - y0 * y0;
        }
        if (ok) {
            float v[4];
            draw4f(k0, k1, link, sweep, (uint32_t)(1024 * sub + 2 * a + 1), v);
            const float ct = 2.0f * v[0] - 1.0f;
            const float st = sqrtf(fmaxf(1.0f - ct * ct, 0.0f));
            float sp, cp;
            sincospif(2.0f * v[1], &sp, &cp);
            const float rr = sqrtf(fmaxf(1.0f - y0 * y0, 0.0f));
            y[0] = y0;
            y[1] = rr * st * cp;
            y[2] = rr * st * sp;
            y[3] = rr * ct;
            return;
        }
    }
    y[0] = 1.0f;
    y[1] = y[2] = y[3] = 0.0f;
}

// rows i, j of w and of the link u (both FP32 here) <- R (rows i, j)
template <int MODE, int I, int J>
__device__ __forceinline__ void subgroup32(cx<float>* u, cx<float>* w, float beta23, uint32_t k0, uint32_t k1,
                                           uint32_t link, uint32_t sweep, int sub)
{
    using F = cx<float>;
    const F wii = w[3 * I + I], wjj = w[3 * J + J], wij = w[3 * I + J], wji = w[3 * J + I];
    const F r = mk(0.5f * (wii.re + wjj.re), 0.5f * (wii.im - wjj.im));
    const F s = mk(0.5f * (wij.re - wji.re), 0.5f * (wij.im + wji.im));
    const float k2 = r.re * r.re + r.im * r.im + s.re * s.re + s.im * s.im;
    if (!(k2 > 0)) return;
    const float ik = rsqrtf(k2);
    const F a = r * ik, b = s * ik;
    F R00, R01, R10, R11;
    if (MODE == 0) {
        float y[4];
        su2_draw_f(beta23 * (k2 * ik), k0, k1, link, sweep, sub, y);
        const F Y00 = mk(y[0], y[3]), Y01 = mk(y[2], y[1]), Y10 = mk(-y[2], y[1]), Y11 = mk(y[0], -y[3]);
        const F nb = mk(-b.re, -b.im);
        R00 = cmac(cmul(Y00, conjg(a)), Y01, conjg(b));
        R01 = cmac(cmul(Y00, nb), Y01, a);
        R10 = cmac(cmul(Y10, conjg(a)), Y11, conjg(b));
        R11 = cmac(cmul(Y10, nb), Y11, a);
    } else {
        const F D00 = conjg(a), D01 = mk(-b.re, -b.im), D10 = conjg(b), D11 = a;
        R00 = cmac(cmul(D00, D00), D01, D10);
        R01 = cmac(cmul(D00, D01), D01, D11);
        R10 = cmac(cmul(D10, D00), D11, D10);
        R11 = cmac(cmul(D10, D01), D11, D11);
    }
    rot_rows<I, J>(w, R00, R01, R10, R11);
    rot_rows<I, J>(u, R00, R01, R10, R11);
}

// U32: an FP32 copy of rows 0,1 of every link ([mu][6][V]), read for the staples
// and kept up to date with the links this launch writes.
template <int MODE>
__global__ void __launch_bounds__(kWilsonThreads) k_wilson32(Lat d, double2* __restrict__ U, float2* __restrict__ U32,
                                                             int mu, int parity, float beta, uint32_t k0, uint32_t k1,
                                                             uint32_t sweep)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= (d.V >> 1)) return;
    const int hx = d.L[0] >> 1;
    int c[4];
    int r = h / hx;
    const int xh = h - r * hx;
    c[1] = r % d.L[1];
    r /= d.L[1];
    c[2] = r % d.L[2];
    c[3] = r / d.L[2];
    c[0] = 2 * xh + ((parity + c[1] + c[2] + c[3]) & 1);
    const int s = c[0] + d.stride[1] * c[1] + d.stride[2] * c[2] + d.stride[3] * c[3];
    const int V = d.V, ne = d.ne;
    cx<float> A[9], uf[9], w[9];
    {
        Lat d32 = d;
        d32.ne = 6;
        staple_sum<float>(d32, U32, mu, s, c, A);
    }
    // the link itself from the FP32 copy, row 2 rebuilt in FP32
    load3<float>(U32, V, 6, mu, s, uf);
    mm<float>(uf, A, w);
    const uint32_t link = (uint32_t)mu * (uint32_t)V + (uint32_t)s;
    const float beta23 = beta * (2.0f / 3.0f);
    subgroup32<MODE, 0, 1>(uf, w, beta23, k0, k1, link, sweep, 0);
    subgroup32<MODE, 0, 2>(uf, w, beta23, k0, k1, link, sweep, 1);
    subgroup32<MODE, 1, 2>(uf, w, beta23, k0, k1, link, sweep, 2);
    // back to FP64 and onto SU(3) there: the stored link is unitary to FP64 rounding
    C u[9];
#pragma unroll
    for (int e = 0; e < 6; e++) u[e] = mk((double)uf[e].re, (double)uf[e].im);
    orthonormal_rows01(u);
#pragma unroll
    for (int e = 0; e < 6; e++) {
        st<double>(U + (size_t)(mu * ne + e) * V + s, u[e]);
        U32[(size_t)(mu * 6 + e) * V + s] = make_float2((float)u[e].re, (float)u[e].im);
    }
    if (ne == 9) {
        complete_row2(u, u + 6);
#pragma unroll
        for (int e = 6; e < 9; e++) st<double>(U + (size_t)(mu * 9 + e) * V + s, u[e]);
    }
}

// the FP32 copy of rows 0,1 of every link
__global__ void k_links_to_fp32(Lat d, const double2* __restrict__ U, float2* __restrict__ U32)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.V) return;
    for (int mu = 0; mu < 4; mu++)
#pragma unroll
        for (int e = 0; e < 6; e++) {
            const double2 v = U[(size_t)(mu * d.ne + e) * d.V + s];
            U32[(size_t)(mu * 6 + e) * d.V + s] = make_float2((float)v.x, (float)v.y);
        }
}

// ---------------------------------------------------------------- plaquette

// Per block: sum over its sites of sum_{mu<nu} Re Tr[U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^dag].
__global__ void __launch_bounds__(kPlaqThreads) k_plaq_partial(Lat d, const double2* __restrict__ U,
                                                              double* __restrict__ part)
{
    double acc = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.V; s += gridDim.x * blockDim.x) {
        int c[4];
        site_coords(d, s, c);
        for (int mu = 0; mu < 3; mu++) {
            const int sp = site_shift(d, s, c[mu], mu, +1);
            for (int nu = mu + 1; nu < 4; nu++) {
                const int sn = site_shift(d, s, c[nu], nu, +1);
                C a[9], b[9], p1[9], p2[9];
                load3<double>(U, d.V, d.ne, mu, s, a);
                load3<double>(U, d.V, d.ne, nu, sp, b);
                mm<double>(a, b, p1);
                load3<double>(U, d.V, d.ne, nu, s, a);
                load3<double>(U, d.V, d.ne, mu, sn, b);
                mm<double>(a, b, p2);
#pragma unroll
                for (int e = 0; e < 9; e++) acc += p1[e].re * p2[e].re + p1[e].im * p2[e].im;
            }
        }
    }
    __shared__ double red[kPlaqThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kPlaqThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out = (sum of the n partials in a fixed order) * scale
__global__ void __launch_bounds__(kPlaqThreads) k_plaq_final(int n, const double* __restrict__ part, double scale,
                                                            double* __restrict__ out)
{
    __shared__ double red[kPlaqThreads];
    double acc = 0;
    for (int i = threadIdx.x; i < n; i += kPlaqThreads) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kPlaqThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

// U_mu(x) = 1 in every stored plane
__global__ void k_unit_links(Lat d, double2* __restrict__ U)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.V) return;
    for (int mu = 0; mu < 4; mu++)
        for (int e = 0; e < d.ne; e++)
            U[(size_t)(mu * d.ne + e) * d.V + s] = make_double2((e == 0 || e == 4 || e == 8) ? 1.0 : 0.0, 0.0);
}

}  // namespace

void launch_unit_links(cudaStream_t s, const Lat& d, double2* U)
{
    k_unit_links<<<(unsigned)((d.V + 255) / 256), 256, 0, s>>>(d, U);
}

int plaquette_blocks(int V)
{
    const int nb = (V + kPlaqThreads - 1) / kPlaqThreads;
    return nb < kPlaqBlocks ? nb : kPlaqBlocks;
}

void launch_links_to_fp32(cudaStream_t s, const Lat& d, const double2* U, float2* U32)
{
    k_links_to_fp32<<<(unsigned)((d.V + 255) / 256), 256, 0, s>>>(d, U, U32);
}

void launch_wilson(cudaStream_t s, const Lat& d, double2* U, float2* U32, int mu, int parity, int overrelax,
                   double beta, unsigned long long seed, unsigned int sweep, int precision)
{
    const unsigned nb = (unsigned)((d.V / 2 + kWilsonThreads - 1) / kWilsonThreads);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    if (precision == 32) {
        if (overrelax)
            k_wilson32<1><<<nb, kWilsonThreads, 0, s>>>(d, U, U32, mu, parity, (float)beta, k0, k1, sweep);
        else
            k_wilson32<0><<<nb, kWilsonThreads, 0, s>>>(d, U, U32, mu, parity, (float)beta, k0, k1, sweep);
    } else if (overrelax) {
        k_wilson<1><<<nb, kWilsonThreads, 0, s>>>(d, U, mu, parity, beta, k0, k1, sweep);
    } else {
        k_wilson<0><<<nb, kWilsonThreads, 0, s>>>(d, U, mu, parity, beta, k0, k1, sweep);
    }
}

void launch_plaquette(cudaStream_t s, const Lat& d, const double2* U, double* part, double* out)
{
    const int nb = plaquette_blocks(d.V);
    k_plaq_partial<<<nb, kPlaqThreads, 0, s>>>(d, U, part);
    k_plaq_final<<<1, kPlaqThreads, 0, s>>>(nb, part, 1.0 / (18.0 * (double)d.V), out);
}

}  // namespace lgf
