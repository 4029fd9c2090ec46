// Shared device-side definitions of the CUDA gauge-fixing library: complex
// arithmetic in registers, SU(3) helpers on the 12-real representation, the
// lattice descriptor and the loop-control block.
//
// Method: Fourier-accelerated steepest descent for Landau gauge, arXiv:1301.3460
// (functional in the introduction; alpha = 0.08 and theta < 1e-15 in the
// description of the 32^4 runs; 12-real link storage named in the GPU set-up).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lgf {

// ---------------------------------------------------------------- complex

template <typename T> struct vec2;
template <> struct vec2<double> { using type = double2; };
template <> struct vec2<float> { using type = float2; };
template <typename T> using vec2_t = typename vec2<T>::type;

template <typename T> struct cx {
    T re, im;
};

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) { return cx<T>{r, i}; }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <typename T> __host__ __device__ __forceinline__ cx<T> conjg(cx<T> a) { return {a.re, -a.im}; }
// a * b
template <typename T> __host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
// a * conj(b)
template <typename T> __host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b)
{
    return {fma(a.re, b.re, a.im * b.im), fma(a.im, b.re, -a.re * b.im)};
}
// acc + a * b
template <typename T> __host__ __device__ __forceinline__ cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + a * conj(b)
template <typename T> __host__ __device__ __forceinline__ cx<T> cmacc(cx<T> acc, cx<T> a, cx<T> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.im, b.re, acc.im);
    acc.im = fma(-a.re, b.im, acc.im);
    return acc;
}
// -i * a and +i * a
template <typename T> __host__ __device__ __forceinline__ cx<T> mul_mi(cx<T> a) { return {a.im, -a.re}; }
template <typename T> __host__ __device__ __forceinline__ cx<T> mul_pi(cx<T> a) { return {-a.im, a.re}; }
template <typename T> __host__ __device__ __forceinline__ T norm2(cx<T> a) { return fma(a.re, a.re, a.im * a.im); }

template <typename T> __device__ __forceinline__ cx<T> ld(const vec2_t<T>* p)
{
    vec2_t<T> v = __ldg(p);
    return {v.x, v.y};
}
template <typename T> __device__ __forceinline__ cx<T> ldv(const vec2_t<T>* p)  // plain load (data written this launch)
{
    vec2_t<T> v = *p;
    return {v.x, v.y};
}
template <typename T> __device__ __forceinline__ void st(vec2_t<T>* p, cx<T> a)
{
    vec2_t<T> v;
    v.x = a.re;
    v.y = a.im;
    *p = v;
}

// ---------------------------------------------------------------- precision conversions

// float -> double (exact) and double -> float (round to nearest, ties to even)
// by integer operations on the IEEE 754 encodings (binary32: sign, 8-bit
// exponent biased by 127, 23-bit fraction; binary64: sign, 11-bit exponent
// biased by 1023, 52-bit fraction).  On this GPU the hardware conversions issue
// on the FP64 pipe (2 per cycle per SM); these use the integer pipe.  Finite
// normal values of the target format take the integer path; zeros, subnormals,
// overflow, infinities and NaNs take the hardware conversion, so every result is
// the hardware's.
__device__ __forceinline__ double f2d_int(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e - 1u >= 254u) return (double)f;
    // exponent rebiased by 1023 - 127; the fraction's top 20 bits in the high
    // word, its low 3 bits at the top of the low word
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ float d2f_int(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned E = (hi >> 20) & 0x7ffu;
    // binary32 exponent E - 896 must lie in [1, 254]
    if (E - 897u >= 254u) return __double2float_rn(x);
    const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the kept 23 fraction bits
    const unsigned rest = lo & 0x1fffffffu;                      // the 29 dropped bits
    unsigned r = (hi & 0x80000000u) | ((E - 896u) << 23) | m23;
    // +1 when rest > 2^28, or rest = 2^28 and m23 is odd; a carry out of the
    // fraction increments the exponent (to infinity from the largest binade)
    r += (rest + 0x0fffffffu + (m23 & 1u)) >> 29;
    return __uint_as_float(r);
}

// ---------------------------------------------------------------- SU(3)

// conj(a b - c d) with four fused multiply-adds per component
template <typename T> __host__ __device__ __forceinline__ cx<T> cdet2c(cx<T> a, cx<T> b, cx<T> c, cx<T> d)
{
    T re = a.re * b.re;
    re = fma(-a.im, b.im, re);
    re = fma(-c.re, d.re, re);
    re = fma(c.im, d.im, re);
    T im = -a.re * b.im;
    im = fma(-a.im, b.re, im);
    im = fma(c.re, d.im, im);
    im = fma(c.im, d.re, im);
    return {re, im};
}

// third row of an SU(3) matrix from its first two (m[0..2] row 0, m[3..5] row 1):
// r2 = conj(r0 x r1)
template <typename T> __host__ __device__ __forceinline__ void complete_row2(const cx<T>* m, cx<T>* r2)
{
    r2[0] = cdet2c(m[1], m[5], m[2], m[4]);
    r2[1] = cdet2c(m[2], m[3], m[0], m[5]);
    r2[2] = cdet2c(m[0], m[4], m[1], m[3]);
}

// 8-real form of an SU(3) matrix: u01, u02, u10 and the phases of u00 and u20.
// Unitarity and det = 1 give the rest: |u00|^2 = 1 - n2 with n2 = |u01|^2 +
// |u02|^2, |u20|^2 = n2 - |u10|^2 (column 0 normalised); rows 0 and 1 orthogonal
// and conj(row0 x row1) = row 2 are two linear equations for u11, u12 with
// determinant n2:
//   u11 = -(t u01 + conj(u02 u20)) / n2,  u12 = (conj(u01 u20) - u02 t) / n2,
//   t = u10 conj(u00);
// row 2 is then rebuilt as conj(row0 x row1).  Singular where n2 = 0 (|u00| = 1).
template <typename T>
__device__ __forceinline__ void rebuild8(cx<T> a01, cx<T> a02, cx<T> a10, T th0, T th2, cx<T>* u)
{
    const T n2 = norm2(a01) + norm2(a02);
    const T m00 = sqrt(fmax(T(1) - n2, T(0)));
    const T m20 = sqrt(fmax(n2 - norm2(a10), T(0)));
    T s0, c0, s2, c2;
    sincos(th0, &s0, &c0);
    sincos(th2, &s2, &c2);
    const cx<T> u00 = mk(m00 * c0, m00 * s0), u20 = mk(m20 * c2, m20 * s2);
    const T inv = T(1) / n2;
    const cx<T> t = cmulc(a10, u00);
    u[0] = u00;
    u[1] = a01;
    u[2] = a02;
    u[3] = a10;
    u[4] = (cmul(t, a01) + conjg(cmul(a02, u20))) * (-inv);
    u[5] = (conjg(cmul(a01, u20)) - cmul(a02, t)) * inv;
    complete_row2(u, u + 6);
}

// ---------------------------------------------------------------- lattice

// Division by a run-time constant d (1 <= d < 2^16) as a multiply-high and a
// shift, exact for numerators 0 <= n < 2^31: s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1, n / d = (umulhi(n, m) + n) >> s.
struct FastDiv {
    unsigned m, s, d;
};
__host__ __device__ inline FastDiv make_fastdiv(unsigned d)
{
    unsigned s = 0;
    while ((1u << s) < d) s++;
    const unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1ull;
    return FastDiv{(unsigned)m, s, d};
}
__host__ __device__ __forceinline__ unsigned fdiv(unsigned n, FastDiv f)
{
#ifdef __CUDA_ARCH__
    const unsigned hi = __umulhi(n, f.m);
#else
    const unsigned hi = (unsigned)(((unsigned long long)n * f.m) >> 32);
#endif
    return (unsigned)(((unsigned long long)hi + n) >> f.s);
}

// Site index s = x + Lx*(y + Ly*(z + Lz*t)).  An xy-plane is the Lx*Ly block of
// one (z, t); plane index p = z + Lz*t.
struct Lat {
    int L[4];
    int stride[4];  // 1, Lx, Lx*Ly, Lx*Ly*Lz
    int V;
    int P;         // Lx*Ly
    int nplanes;   // Lz*Lt
    int ne;        // complex entries stored per link: 6 (rows 0,1; row 2 rebuilt on load),
                   // 9 (row 2 kept as written, the rebuild done once when stored) or
                   // 4 (the 8-real form, FP64 only: u01, u02, u10, phases of u00 and u20)
    FastDiv dLx, dLy, dP;  // division by Lx, Ly and Lx*Ly
};

// the division helpers of a lattice descriptor (call after L is set)
inline void lat_set_divisors(Lat& d)
{
    d.dLx = make_fastdiv((unsigned)d.L[0]);
    d.dLy = make_fastdiv((unsigned)d.L[1]);
    d.dP = make_fastdiv((unsigned)(d.L[0] * d.L[1]));
}

__device__ __forceinline__ int site_shift(const Lat& d, int s, int c_mu, int mu, int dir)
{
    // c_mu is the mu coordinate of s; dir = +1 or -1 with periodic wrap
    if (dir > 0) return (c_mu == d.L[mu] - 1) ? s - (d.L[mu] - 1) * d.stride[mu] : s + d.stride[mu];
    return (c_mu == 0) ? s + (d.L[mu] - 1) * d.stride[mu] : s - d.stride[mu];
}

__device__ __forceinline__ void site_coords(const Lat& d, int s, int c[4])
{
    c[0] = s % d.L[0];
    int r = s / d.L[0];
    c[1] = r % d.L[1];
    r /= d.L[1];
    c[2] = r % d.L[2];
    c[3] = r / d.L[2];
}

// ---------------------------------------------------------------- control

// Device-resident loop state of one gauge fixing.  The Delta kernel's last
// block writes theta and F and decides whether the running loop stops.
struct Ctl {
    double theta;          // of the current links
    double F;
    double tol;            // stop threshold of the running phase
    double tol_final;      // threshold of the FP64 phase
    double alpha;          // steepest-descent step
    int iter;              // updates applied (all phases)
    int max_iter;
    int phase;             // 0: FP32 phase of the mixed mode, 1: FP64
    int phase_done;        // the running loop has met its stop condition
    int done;              // the whole fix is over
    int converged;
    int nan_seen;
    int iter_phase0;       // updates applied in the FP32 phase
    unsigned int ticket;   // last-block counter of the reduction
    unsigned int body_runs;
    int hist_cap;
    unsigned int loop_bound;  // extra cap on body runs of a device loop (0: none)
    double theta_best;     // smallest theta of the FP32 phase so far
    int iter_best;         // the iteration that reached it
    int stall;             // FP32 phase ends after this many iterations without a new smallest theta (0: never) ...
    int stall_near;        // ... or after this many once theta_best < near_floor
    double near_floor;
    int fault;             // a kernel gave up waiting for its own asynchronous copies (loop stopped)
};

}  // namespace lgf
