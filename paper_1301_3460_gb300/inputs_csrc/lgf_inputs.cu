// Seeded synthetic SU(3) gauge fields drawn on the GPU, for ensembles too large
// to draw on the host.  Input generation only: this library shares no code with
// the gauge-fixing kernels and computes none of the method's steps.
//
//   U_mu(x) = h(x) exp(i eps A_mu(x)) h^dag(x+mu)
//
// * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
//   numbers: as easy as 1, 2, 3", SC'11), counter = (index, draw, 0, 0), key =
//   the seed; uniforms in (0, 1] from 32-bit words, Gaussians by Box-Muller.
// * h(x): the Q of a complex Gaussian 3x3 matrix with R's diagonal made
//   positive (Haar measure on U(3), Mezzadri's recipe), by modified Gram-Schmidt
//   on columns with re-orthogonalisation, then multiplied by a cube root of
//   conj(det) to land in SU(3).
// * A_mu(x) = sum_a w_a lambda_a / 2 with w_a ~ N(0, 1); the exponential by a
//   12th-order Taylor polynomial of the matrix scaled by 2^-s, squared s times.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

struct c2 {
    double re, im;
};
__device__ __forceinline__ c2 add(c2 a, c2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ c2 sub(c2 a, c2 b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ c2 mul(c2 a, c2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ c2 cmulconj(c2 a, c2 b) { return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im}; }  // conj(b) a
__device__ __forceinline__ c2 scale(c2 a, double s) { return {a.re * s, a.im * s}; }

__device__ __forceinline__ void philox(uint32_t ctr[4], uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(M0, ctr[0]), lo0 = M0 * ctr[0];
        const uint32_t hi1 = __umulhi(M1, ctr[2]), lo1 = M1 * ctr[2];
        const uint32_t n0 = hi1 ^ ctr[1] ^ k0, n2 = hi0 ^ ctr[3] ^ k1;
        ctr[0] = n0;
        ctr[1] = lo1;
        ctr[2] = n2;
        ctr[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// four standard normals for (index, draw)
__device__ __forceinline__ void normals4(uint64_t seed, uint64_t index, uint32_t draw, double out[4])
{
    uint32_t c[4] = {(uint32_t)index, (uint32_t)(index >> 32), draw, 0u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double two_pi = 6.283185307179586476925286766559;
    for (int p = 0; p < 2; p++) {
        const double u1 = ((double)c[2 * p] + 1.0) * 2.3283064365386962890625e-10;  // (0, 1]
        const double u2 = (double)c[2 * p + 1] * 2.3283064365386962890625e-10;       // [0, 1)
        const double r = sqrt(-2.0 * log(u1));
        double s, co;
        sincos(two_pi * u2, &s, &co);
        out[2 * p] = r * co;
        out[2 * p + 1] = r * s;
    }
}

__device__ void haar_su3(uint64_t seed, uint64_t site, c2* q /* 9, row-major */)
{
    double g[20];
    for (int d = 0; d < 5; d++) normals4(seed, site, (uint32_t)d, g + 4 * d);
    const double is2 = 0.70710678118654752440;
    c2 z[9];
    for (int e = 0; e < 9; e++) z[e] = {g[2 * e] * is2, g[2 * e + 1] * is2};
    // modified Gram-Schmidt on the columns of z, each projection done twice so
    // that ill-conditioned draws still give columns orthonormal to rounding
    for (int j = 0; j < 3; j++) {
        for (int pass = 0; pass < 2; pass++)
            for (int k = 0; k < j; k++) {
                c2 ip = {0, 0};
                for (int i = 0; i < 3; i++) ip = add(ip, cmulconj(z[3 * i + j], q[3 * i + k]));
                for (int i = 0; i < 3; i++) z[3 * i + j] = sub(z[3 * i + j], mul(ip, q[3 * i + k]));
            }
        double n = 0;
        for (int i = 0; i < 3; i++) n += z[3 * i + j].re * z[3 * i + j].re + z[3 * i + j].im * z[3 * i + j].im;
        n = 1.0 / sqrt(n);
        for (int i = 0; i < 3; i++) q[3 * i + j] = scale(z[3 * i + j], n);
    }
    // det q = e^{i phi}; multiply by e^{-i phi/3}
    c2 det = add(add(mul(q[0], sub(mul(q[4], q[8]), mul(q[5], q[7]))),
                     scale(mul(q[1], sub(mul(q[3], q[8]), mul(q[5], q[6]))), -1.0)),
                 mul(q[2], sub(mul(q[3], q[7]), mul(q[4], q[6]))));
    const double phi = atan2(det.im, det.re) / 3.0;
    double s, co;
    sincos(-phi, &s, &co);
    const c2 f = {co, s};
    for (int e = 0; e < 9; e++) q[e] = mul(q[e], f);
}

__device__ void matmul(const c2* a, const c2* b, c2* c)
{
    c2 t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            c2 acc = {0, 0};
            for (int k = 0; k < 3; k++) acc = add(acc, mul(a[3 * i + k], b[3 * k + j]));
            t[3 * i + j] = acc;
        }
    for (int e = 0; e < 9; e++) c[e] = t[e];
}

// exp(i eps A) for A = sum_a w_a lambda_a / 2
__device__ void exp_i_eps_A(const double* w, double eps, c2* E)
{
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    // A (Hermitian), times i eps: X = i eps A
    c2 A[9];
    A[0] = {0.5 * (w[2] + r3 * w[7]), 0};
    A[4] = {0.5 * (-w[2] + r3 * w[7]), 0};
    A[8] = {-r3 * w[7], 0};
    A[1] = {0.5 * w[0], -0.5 * w[1]};
    A[3] = {0.5 * w[0], 0.5 * w[1]};
    A[2] = {0.5 * w[3], -0.5 * w[4]};
    A[6] = {0.5 * w[3], 0.5 * w[4]};
    A[5] = {0.5 * w[5], -0.5 * w[6]};
    A[7] = {0.5 * w[5], 0.5 * w[6]};
    double nrm = 0;
    for (int e = 0; e < 9; e++) nrm += A[e].re * A[e].re + A[e].im * A[e].im;
    nrm = sqrt(nrm) * fabs(eps);
    int s = 0;
    while (nrm > 0.25 && s < 30) {
        nrm *= 0.5;
        s++;
    }
    const double sc = eps * ldexp(1.0, -s);
    c2 X[9];
    for (int e = 0; e < 9; e++) X[e] = {-A[e].im * sc, A[e].re * sc};  // i * sc * A
    // Horner: E = I + X/1 (I + X/2 (I + ... (I + X/12)))
    for (int e = 0; e < 9; e++) E[e] = {(e % 4 == 0) ? 1.0 : 0.0, 0};
    for (int k = 12; k >= 1; k--) {
        c2 T[9];
        matmul(X, E, T);
        for (int e = 0; e < 9; e++) E[e] = scale(T[e], 1.0 / k);
        E[0].re += 1.0;
        E[4].re += 1.0;
        E[8].re += 1.0;
    }
    for (int i = 0; i < s; i++) matmul(E, E, E);
}

__global__ void k_haar(int V, uint64_t seed, double* h /* [V][3][3] complex */)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    c2 q[9];
    haar_su3(seed, (uint64_t)s, q);
    for (int e = 0; e < 9; e++) {
        h[(size_t)s * 18 + 2 * e] = q[e].re;
        h[(size_t)s * 18 + 2 * e + 1] = q[e].im;
    }
}

__global__ void k_links(int Lx, int Ly, int Lz, int Lt, double eps, uint64_t seed, int haar, const double* h,
                        double* U /* [4][V][3][3] complex */)
{
    const long V = (long)Lx * Ly * Lz * Lt;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * V) return;
    const int mu = (int)(idx / V);
    const long s = idx - (long)mu * V;
    double w[8];
    double g[8];
    normals4(seed ^ 0x5bd1e9955bd1e995ull, (uint64_t)idx, 0u, g);
    normals4(seed ^ 0x5bd1e9955bd1e995ull, (uint64_t)idx, 1u, g + 4);
    for (int a = 0; a < 8; a++) w[a] = g[a];
    c2 W[9];
    exp_i_eps_A(w, eps, W);
    if (haar) {
        const int L[4] = {Lx, Ly, Lz, Lt};
        long st = 1;
        for (int nu = 0; nu < mu; nu++) st *= L[nu];
        const long c = (s / st) % L[mu];
        const long sn = (c == L[mu] - 1) ? s - (long)(L[mu] - 1) * st : s + st;
        c2 hx[9], hn[9], T[9];
        for (int e = 0; e < 9; e++) {
            hx[e] = {h[s * 18 + 2 * e], h[s * 18 + 2 * e + 1]};
            hn[e] = {h[sn * 18 + 2 * e], h[sn * 18 + 2 * e + 1]};
        }
        matmul(hx, W, T);
        // W = T hn^dag
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                c2 acc = {0, 0};
                for (int k = 0; k < 3; k++) acc = add(acc, cmulconj(T[3 * i + k], hn[3 * j + k]));
                W[3 * i + j] = acc;
            }
    }
    for (int e = 0; e < 9; e++) {
        U[idx * 18 + 2 * e] = W[e].re;
        U[idx * 18 + 2 * e + 1] = W[e].im;
    }
}

}  // namespace

// U_out: device [4][V][3][3] complex128; h_scratch: device [V][3][3] complex128
// (caller-provided; unused when haar = 0).  Returns 0 or a cudaError_t value.
extern "C" int lgf_inputs_rough_field(const int dims[4], double eps, unsigned long long seed, int haar,
                                      double* h_scratch, double* U_out, void* stream)
{
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (haar) k_haar<<<(unsigned)((V + 255) / 256), 256, 0, s>>>((int)V, seed, h_scratch);
    k_links<<<(unsigned)((4 * V + 255) / 256), 256, 0, s>>>(dims[0], dims[1], dims[2], dims[3], eps, seed, haar,
                                                         h_scratch, U_out);
    return (int)cudaGetLastError();
}
