// Kernels of one Fourier-accelerated steepest-descent iteration (arXiv:1301.3460):
//
//   k_delta      Delta(x) = (M - M^dag) - Tr(M - M^dag)/3, M = sum_mu [U_mu(x-mu) - U_mu(x)],
//                packed into four complex fields (as sums of the links' packed
//                anti-Hermitian parts), theta and F reduced in FP64, then the
//                forward FFT along x and y of the xy-plane.
//   k_zt         forward FFT along z and t, the accelerator p2max/(p2(k) V)
//                (zero mode removed), inverse FFT along t and z.
//   k_xyinv_g    inverse FFT along x and y, then g(x) = reunit(1 + alpha/2 Delta~(x))
//                by row Gram-Schmidt in FP64.
//   k_update     U_mu(x) <- g(x) U_mu(x) g^dag(x+mu) and G(x) <- g(x) G(x); writes the
//                packed anti-Hermitian parts and Re Tr of the new links for k_delta.
//
// Storage (structure of arrays, one plane of V complex numbers per entry):
//   links U  [mu=4][e=6][V]  rows 0,1 of U_mu(x), e = 3 i + j; row 2 is rebuilt
//                            as conj(row0 x row1) on every load (12-real form)
//   G        [6][V]          rows 0,1 of the accumulated gauge transformation
//   g        [9][V]          the full 3x3 g(x), read by up to nine sites
//   fields   [4][V]          Delta01, Delta02, Delta12 and i*(Im Delta00) + ... packed
//                            as (Im Delta00) + i (Im Delta11)
// Delta is anti-Hermitian and traceless, so these four complex numbers carry
// its eight real degrees of freedom; the accelerator is real and even in k, so
// it maps each packed real pair to a real pair and the packing commutes with it.
#pragma once
#include "lgf_common.cuh"
#include "lgf_fft.cuh"

namespace lgf {

__device__ __forceinline__ int ld_flag(const int* p) { return *(const volatile int*)p; }

// ---------------------------------------------------------------- reductions

constexpr int kMaxThreads = 512;  // block size bound of every plane-tiled kernel

__device__ __forceinline__ double block_sum(double v, double* scratch /* kMaxThreads/32 */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    double r = 0;
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int i = 0; i < nw; i++) r += scratch[i];
    }
    return r;  // valid in thread 0
}

// Per-block partial sums of theta and F, then the last block to finish sums
// the partials in block order (deterministic) and updates the loop state.
static __device__ void reduce_theta_F(double th, double f, double* __restrict__ partials, Ctl* ctl, double2* hist, int V)
{
    __shared__ double scratch[kMaxThreads / 32];
    __shared__ int am_last;
    double bt = block_sum(th, scratch);
    double bf = block_sum(f, scratch);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = bt;
        partials[2 * blockIdx.x + 1] = bf;
        __threadfence();
        unsigned int tk = atomicAdd(&ctl->ticket, 1u);
        am_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double a = 0, b = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(partials + 2 * i);
        b += __ldcg(partials + 2 * i + 1);
    }
    a = block_sum(a, scratch);
    b = block_sum(b, scratch);
    if (threadIdx.x == 0) {
        const double theta = a / (3.0 * (double)V);
        const double F = b / (12.0 * (double)V);
        ctl->theta = theta;
        ctl->F = F;
        const int it = ctl->iter;
        if (hist != nullptr && ctl->hist_cap > 0) hist[it % ctl->hist_cap] = make_double2(theta, F);
        if (!(theta == theta) || !(F == F) || isinf(theta)) {
            ctl->nan_seen = 1;
            ctl->phase_done = 1;
            ctl->done = 1;
        } else if (theta < ctl->tol) {
            ctl->phase_done = 1;
            if (ctl->phase == 1) {
                ctl->done = 1;
                ctl->converged = 1;
            }
        } else if (it >= ctl->max_iter) {
            ctl->phase_done = 1;
            ctl->done = 1;
        } else if (ctl->phase == 0 && ctl->stall > 0) {
            // FP32 arithmetic has stopped improving theta: hand over to FP64
            if (theta < ctl->theta_best) {
                ctl->theta_best = theta;
                ctl->iter_best = it;
            } else if (it - ctl->iter_best >= (ctl->theta_best < ctl->near_floor ? ctl->stall_near : ctl->stall)) {
                ctl->phase_done = 1;
            }
        }
        ctl->ticket = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------- link loads

// link (mu, s), layout [mu][ne][V]: rows 0,1 and row 2 (rebuilt as conj(r0 x r1)
// when ne = 6, read when ne = 9, in which case it was stored as that rebuild), or
// the whole matrix rebuilt from its 8-real form (ne = 4, FP64)
template <typename T>
__device__ __forceinline__ void load_link(const vec2_t<T>* __restrict__ U, int V, int ne, int mu, int s, cx<T>* u)
{
    if constexpr (sizeof(T) == 8) {
        if (ne == 4) {
            const vec2_t<T>* p = U + (size_t)(mu * 4) * V + s;
            const vec2_t<T> th = __ldg(p + 3 * (size_t)V);
            rebuild8<T>(ld<T>(p), ld<T>(p + V), ld<T>(p + 2 * (size_t)V), th.x, th.y, u);
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 6; e++) u[e] = ld<T>(U + (size_t)(mu * ne + e) * V + s);
    if (ne == 9) {
#pragma unroll
        for (int e = 6; e < 9; e++) u[e] = ld<T>(U + (size_t)(mu * 9 + e) * V + s);
    } else {
        complete_row2(u, u + 6);
    }
}

// store link (mu, s) from its full matrix w in the layout of ne (see load_link)
template <typename T>
__device__ __forceinline__ void store_link(vec2_t<T>* __restrict__ U, int V, int ne, int mu, int s, const cx<T>* w)
{
    if constexpr (sizeof(T) == 8) {
        if (ne == 4) {
            vec2_t<T>* p = U + (size_t)(mu * 4) * V + s;
            st<T>(p, w[1]);
            st<T>(p + V, w[2]);
            st<T>(p + 2 * (size_t)V, w[3]);
            vec2_t<T> th;
            th.x = atan2(w[0].im, w[0].re);
            th.y = atan2(w[6].im, w[6].re);
            p[3 * (size_t)V] = th;
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 6; e++) st<T>(U + (size_t)(mu * ne + e) * V + s, w[e]);
    if (ne == 9) {
#pragma unroll
        for (int e = 6; e < 9; e++) st<T>(U + (size_t)(mu * 9 + e) * V + s, w[e]);
    }
}

template <typename T>
__device__ __forceinline__ void load_g(const vec2_t<T>* __restrict__ g, int V, int s, cx<T>* m)
{
#pragma unroll
    for (int e = 0; e < 9; e++) m[e] = ld<T>(g + (size_t)e * V + s);
}

// ---------------------------------------------------------------- k_delta

// The traceless anti-Hermitian part of one link w (full matrix), packed as four
// complex numbers in the layout of the Delta fields: w01 - conj(w10),
// w02 - conj(w20), w12 - conj(w21), and 2 (Im w00 - t) + 2 i (Im w11 - t) with
// t = (Im w00 + Im w11 + Im w22)/3.  Delta(x) is linear in the links, so it is
// the sum over mu of ah(U_mu(x - mu)) - ah(U_mu(x)).
template <typename T> __device__ __forceinline__ void ah_pack(const cx<T>* w, cx<T>* a)
{
    a[0] = w[1] - conjg(w[3]);
    a[1] = w[2] - conjg(w[6]);
    a[2] = w[5] - conjg(w[7]);
    const T t = (w[0].im + w[4].im + w[8].im) * (T)(1.0 / 3.0);
    a[3] = mk<T>((T)2 * (w[0].im - t), (T)2 * (w[4].im - t));
}

// ah of every link and the per-site sum of Re Tr over the four links, from
// links whose row 2 is rebuilt (before the first iteration; the update kernel
// writes them for the links it produces).  AH: [mu=4][k=4][V], Fs: [V].
template <typename T>
__global__ void __launch_bounds__(256) k_ah_init(Lat d, const vec2_t<T>* __restrict__ U, vec2_t<T>* __restrict__ AH,
                                                 T* __restrict__ Fs)
{
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    T f = 0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<T> u[9], a[4];
        load_link<T>(U, V, d.ne, mu, s, u);
        ah_pack(u, a);
#pragma unroll
        for (int k = 0; k < 4; k++) st<T>(AH + (size_t)(mu * 4 + k) * V + s, a[k]);
        f += u[0].re + u[4].re + u[8].re;
    }
    Fs[s] = f;
}

// One block per xy-plane.  Shared memory: (4 + nfc) * P complex values.
// Delta(x) = sum_mu ah_mu(x - mu) - ah_mu(x) (packed fields), theta and F
// reduced in FP64, then (FFT = true) the forward FFT along x and y.
template <typename T, bool FFT>
__global__ void __launch_bounds__(kMaxThreads) k_delta(Lat d, const XyFft F, const vec2_t<T>* __restrict__ AH,
                                                       const T* __restrict__ Fs, vec2_t<T>* __restrict__ Fd,
                                                       double* __restrict__ partials, Ctl* ctl, double2* hist,
                                                       const vec2_t<T>* __restrict__ twx,
                                                       const vec2_t<T>* __restrict__ twy)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    if (ld_flag(&ctl->phase_done)) return;
    const int P = d.P, V = d.V;
    const int plane = blockIdx.x;
    const int s0 = plane * P;
    const int z = plane % d.L[2], t = plane / d.L[2];
    double th = 0.0, fsum = 0.0;
#pragma unroll 4
    for (int xy = threadIdx.x; xy < P; xy += blockDim.x) {
        const int s = s0 + xy;
        const int x = xy % d.L[0], y = xy / d.L[0];
        const int c[4] = {x, y, z, t};
        cx<T> D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) D[k] = mk<T>(0, 0);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const int sb = site_shift(d, s, c[mu], mu, -1);
#pragma unroll
            for (int k = 0; k < 4; k++)
                D[k] = D[k] + ld<T>(AH + (size_t)(mu * 4 + k) * V + sb) - ld<T>(AH + (size_t)(mu * 4 + k) * V + s);
        }
        fsum += (double)__ldg(Fs + s);
        const T a = D[3].re, b = D[3].im, cc = a + b;
        // per-site sum of |Delta_ij|^2 in the kernel's precision, accumulated over
        // sites in FP64
        th += (double)((T)2 * (norm2(D[0]) + norm2(D[1]) + norm2(D[2])) + a * a + b * b + cc * cc);
#pragma unroll
        for (int k = 0; k < 4; k++) st<T>(sm + k * P + xy, D[k]);
    }
    reduce_theta_F(th, fsum, partials, ctl, hist, V);
    __syncthreads();
    // forward FFT along x (lines: fields x Ly rows) and along y (fields x Lx columns)
    if (FFT) fft_xy_fields<T>(F, P, sm, sm + 4 * P, twx, twy, kFwd);
    for (int i = threadIdx.x; i < 4 * P; i += blockDim.x) {
        const int f = i / P, xy = i - f * P;
        Fd[(size_t)f * V + s0 + xy] = sm[i];
    }
}

// ---------------------------------------------------------------- k_zt

// One block per (x-chunk of xw columns, y, field).  Shared memory: two buffers of
// Lt rows of Z.rs >= xw * Lz values, laid out [t][z][xi].  Data arrive transformed along x and
// y, so the x and y indices are the momenta kx, ky.
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) k_zt(Lat d, const ZtFft Z, vec2_t<T>* __restrict__ Fd, const Ctl* ctl,
                                                    const vec2_t<T>* __restrict__ twz,
                                                    const vec2_t<T>* __restrict__ twt, const T* __restrict__ mult,
                                                    const double* __restrict__ s2x, const double* __restrict__ s2y,
                                                    const double* __restrict__ s2z, const double* __restrict__ s2t,
                                                    double p2max)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    if (ld_flag(&ctl->phase_done)) return;
    const int XW = Z.xw, RS = Z.rs;
    const int Lz = d.L[2], Lt = d.L[3], P = d.P;
    const int x0 = blockIdx.x * XW, y = blockIdx.y, f = blockIdx.z;
    vec2_t<T>* base = Fd + (size_t)f * d.V + x0 + d.L[0] * y;
    const int n = XW * Lz * Lt;
    const int LzXW = Lz * XW;
    // value i = xi + XW (z + Lz t) of the pencil sits at t RS + (i mod Lz XW) in the tile
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int zt = i / XW, xi = i - zt * XW;
        const int t = i / LzXW;
        sm[i + t * (RS - LzXW)] = base[xi + (size_t)P * zt];
    }
    __syncthreads();
    vec2_t<T>* a = sm;
    vec2_t<T>* b = sm + (size_t)Lt * RS;
    // forward along z and t
    vec2_t<T>* r = fft_lines<T>(Z.pz, a, b, Z.lz, 1, Z.mz, twz, kFwd);
    r = fft_lines<T>(Z.pt, r, r == a ? b : a, Z.lt, 1, Z.mt, twt, kFwd);
    // the accelerator p2max / (p2(k) V), zero mode removed: from the table of
    // multipliers (site-indexed by momentum) when there is one, else computed
    if (mult != nullptr) {
        const T* mrow = mult + x0 + d.L[0] * y;
#pragma unroll 4
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int zt = i / XW, xi = i - zt * XW;
            const int o = i + (i / LzXW) * (RS - LzXW);
            const T m = __ldg(mrow + xi + (size_t)P * zt);
            vec2_t<T> v = r[o];
            v.x *= m;
            v.y *= m;
            r[o] = v;
        }
    } else {
        const double inv_v = 1.0 / (double)d.V;
        const double sy = s2y[y];
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int zt = i / XW, xi = i - zt * XW;
            const int kt = zt / Lz, kz = zt - kt * Lz;
            const double p2 = s2x[x0 + xi] + sy + s2z[kz] + s2t[kt];
            const T m = (p2 > 0.0) ? (T)(p2max / p2 * inv_v) : (T)0;
            const int o = i + kt * (RS - LzXW);
            vec2_t<T> v = r[o];
            v.x *= m;
            v.y *= m;
            r[o] = v;
        }
    }
    __syncthreads();
    // inverse along t and z
    r = fft_lines<T>(Z.pt, r, r == a ? b : a, Z.lt, 1, Z.mt, twt, kInv);
    r = fft_lines<T>(Z.pz, r, r == a ? b : a, Z.lz, 1, Z.mz, twz, kInv);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int zt = i / XW, xi = i - zt * XW;
        base[xi + (size_t)P * zt] = r[i + (i / LzXW) * (RS - LzXW)];
    }
}

// multiplier table p2max / (p2(k) V) for every momentum k (site-indexed), FP64 and FP32
static __global__ void k_make_mult(Lat d, const double* __restrict__ s2x, const double* __restrict__ s2y,
                                   const double* __restrict__ s2z, const double* __restrict__ s2t, double p2max,
                                   double* __restrict__ m64, float* __restrict__ m32)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.V) return;
    int c[4];
    site_coords(d, s, c);
    const double p2 = s2x[c[0]] + s2y[c[1]] + s2z[c[2]] + s2t[c[3]];
    const double m = (p2 > 0.0) ? p2max / p2 / (double)d.V : 0.0;
    m64[s] = m;
    m32[s] = (float)m;
}

// ---------------------------------------------------------------- k_xyinv_g

// row Gram-Schmidt of rows 0,1 of X in FP64: the orthonormal rows 0,1 of g
// squared norm of a row of three complex numbers as one multiply and five FMAs
__device__ __forceinline__ double row_norm2(const cx<double>* r)
{
    double n = r[0].re * r[0].re;
    n = fma(r[0].im, r[0].im, n);
    n = fma(r[1].re, r[1].re, n);
    n = fma(r[1].im, r[1].im, n);
    n = fma(r[2].re, r[2].re, n);
    return fma(r[2].im, r[2].im, n);
}

// row Gram-Schmidt of rows 0,1 of X in FP64: the orthonormal rows 0,1 of g
// (every subtraction folded into an FMA: this runs on the 2-per-cycle FP64 pipe)
__device__ __forceinline__ void gram_schmidt01(const cx<double>* X /* 6 in */, cx<double>* g /* 6 out */)
{
    const double n0 = rsqrt(row_norm2(X));
    g[0] = X[0] * n0;
    g[1] = X[1] * n0;
    g[2] = X[2] * n0;
    // <r0, X1> = sum conj(r0_j) X1_j
    cx<double> ip = cmulc(X[3], g[0]);
    ip = cmacc(ip, X[4], g[1]);
    ip = cmacc(ip, X[5], g[2]);
    // r1 = X1 - ip r0
    cx<double> r1[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        r1[j].re = fma(-ip.re, g[j].re, fma(ip.im, g[j].im, X[3 + j].re));
        r1[j].im = fma(-ip.re, g[j].im, fma(-ip.im, g[j].re, X[3 + j].im));
    }
    const double n1 = rsqrt(row_norm2(r1));
    g[3] = r1[0] * n1;
    g[4] = r1[1] * n1;
    g[5] = r1[2] * n1;
}

// all three rows in FP64: row 2 = conj(r0 x r1)
__device__ __forceinline__ void reunit_rows(cx<double>* X /* 6 in */, cx<double>* g /* 9 out */)
{
    gram_schmidt01(X, g);
    complete_row2(g, g + 6);
}

// One block per xy-plane.  g is built in FP64 whatever T is, and stored as TG.
template <typename T, typename TG>
__global__ void __launch_bounds__(kMaxThreads) k_xyinv_g(Lat d, const XyFft F, const vec2_t<T>* __restrict__ Fd,
                                                         vec2_t<TG>* __restrict__ g,
                                                const Ctl* ctl, const vec2_t<T>* __restrict__ twx,
                                                const vec2_t<T>* __restrict__ twy)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    if (ld_flag(&ctl->phase_done)) return;
    const int P = d.P, V = d.V;
    const int s0 = blockIdx.x * P;
#pragma unroll 4
    for (int i = threadIdx.x; i < 4 * P; i += blockDim.x) {
        const int f = i / P, xy = i - f * P;
        sm[i] = Fd[(size_t)f * V + s0 + xy];
    }
    __syncthreads();
    fft_xy_fields<T>(F, P, sm, sm + 4 * P, twx, twy, kInv);
    const double h = 0.5 * ctl->alpha;
    for (int xy = threadIdx.x; xy < P; xy += blockDim.x) {
        vec2_t<T> f0 = sm[xy], f1 = sm[P + xy], f2 = sm[2 * P + xy], f3 = sm[3 * P + xy];
        // X = 1 + (alpha/2) Delta~ ; rows 0 and 1
        cx<double> X[6];
        X[0] = mk<double>(1.0, h * (double)f3.x);
        X[1] = mk<double>(h * (double)f0.x, h * (double)f0.y);
        X[2] = mk<double>(h * (double)f1.x, h * (double)f1.y);
        X[3] = mk<double>(-h * (double)f0.x, h * (double)f0.y);  // -conj(Delta01)
        X[4] = mk<double>(1.0, h * (double)f3.y);
        X[5] = mk<double>(h * (double)f2.x, h * (double)f2.y);
        // Gram-Schmidt in FP64; row 2 = conj(r0 x r1) in the precision g is
        // stored in (for an FP32 g, from the rounded rows, so that the stored g
        // is unitary to FP32 rounding)
        cx<double> gm[6];
        gram_schmidt01(X, gm);
        cx<TG> gs[9];
#pragma unroll
        for (int e = 0; e < 6; e++) gs[e] = mk<TG>((TG)gm[e].re, (TG)gm[e].im);
        complete_row2(gs, gs + 6);
#pragma unroll
        for (int e = 0; e < 9; e++) st<TG>(g + (size_t)e * V + s0 + xy, gs[e]);
    }
}

// g(x) = reunit(1 + alpha/2 D(x)) from the four packed spatial fields D (plain
// steepest descent: the step uses Delta itself), one thread per site
template <typename T, typename TG>
__global__ void __launch_bounds__(256) k_build_g(Lat d, const vec2_t<T>* __restrict__ Fd, vec2_t<TG>* __restrict__ g,
                                                 const Ctl* ctl)
{
    if (ld_flag(&ctl->phase_done)) return;
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const double h = 0.5 * ctl->alpha;
    const vec2_t<T> f0 = Fd[s], f1 = Fd[(size_t)V + s], f2 = Fd[(size_t)2 * V + s], f3 = Fd[(size_t)3 * V + s];
    cx<double> X[6];
    X[0] = mk<double>(1.0, h * (double)f3.x);
    X[1] = mk<double>(h * (double)f0.x, h * (double)f0.y);
    X[2] = mk<double>(h * (double)f1.x, h * (double)f1.y);
    X[3] = mk<double>(-h * (double)f0.x, h * (double)f0.y);
    X[4] = mk<double>(1.0, h * (double)f3.y);
    X[5] = mk<double>(h * (double)f2.x, h * (double)f2.y);
    cx<double> gm[6];
    gram_schmidt01(X, gm);
    cx<TG> gs[9];
#pragma unroll
    for (int e = 0; e < 6; e++) gs[e] = mk<TG>((TG)gm[e].re, (TG)gm[e].im);
    complete_row2(gs, gs + 6);
#pragma unroll
    for (int e = 0; e < 9; e++) st<TG>(g + (size_t)e * V + s, gs[e]);
}

// ---------------------------------------------------------------- k_update

// One thread per site.  G may be null (gauge not tracked).  Also writes the
// packed anti-Hermitian parts of the new links (AH) and their Re Tr per site
// (Fs) for the next Delta.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_update(Lat d, vec2_t<T>* __restrict__ U,
                                                                        vec2_t<T>* __restrict__ G,
                                                                        const vec2_t<T>* __restrict__ g, Ctl* ctl,
                                                                        vec2_t<T>* __restrict__ AH,
                                                                        T* __restrict__ Fs)
{
    if (ld_flag(&ctl->phase_done)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->iter += 1;
        if (ctl->phase == 0) ctl->iter_phase0 += 1;
    }
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    cx<T> gx[9];
    load_g<T>(g, V, s, gx);
    T f = 0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<T> u[9];
        load_link<T>(U, V, d.ne, mu, s, u);
        // A = rows 0,1 of g(x) U
        cx<T> A[6];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<T> acc = cmul(gx[3 * i], u[j]);
                acc = cmac(acc, gx[3 * i + 1], u[3 + j]);
                acc = cmac(acc, gx[3 * i + 2], u[6 + j]);
                A[3 * i + j] = acc;
            }
        cx<T> gn[9];
        load_g<T>(g, V, site_shift(d, s, c[mu], mu, +1), gn);
        // U' = A g^dag(x+mu): U'_ij = sum_k A_ik conj(gn_jk); row 2 rebuilt
        cx<T> w[9];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<T> acc = cmulc(A[3 * i], gn[3 * j]);
                acc = cmacc(acc, A[3 * i + 1], gn[3 * j + 1]);
                acc = cmacc(acc, A[3 * i + 2], gn[3 * j + 2]);
                w[3 * i + j] = acc;
            }
        complete_row2(w, w + 6);
        store_link<T>(U, V, d.ne, mu, s, w);
        cx<T> a[4];
        ah_pack(w, a);
#pragma unroll
        for (int k = 0; k < 4; k++) st<T>(AH + (size_t)(mu * 4 + k) * V + s, a[k]);
        f += w[0].re + w[4].re + w[8].re;
    }
    Fs[s] = f;
    if (G != nullptr) {
        cx<T> Gm[9];
#pragma unroll
        for (int e = 0; e < 6; e++) Gm[e] = ldv<T>(G + (size_t)e * V + s);
        complete_row2(Gm, Gm + 6);
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<T> acc = cmul(gx[3 * i], Gm[j]);
                acc = cmac(acc, gx[3 * i + 1], Gm[3 + j]);
                acc = cmac(acc, gx[3 * i + 2], Gm[6 + j]);
                st<T>(G + (size_t)(3 * i + j) * V + s, acc);
            }
    }
}

// ---------------------------------------------------------------- loop control

// Last node of the while-loop body: keep looping while the running phase has
// not met its stop condition; a hard bound on body runs makes the loop finite
// whatever the state says.
static __global__ void k_loop_ctl(Ctl* ctl, cudaGraphConditionalHandle h, unsigned int bound)
{
    unsigned int n = ctl->body_runs + 1u;
    ctl->body_runs = n;
    const unsigned int cap = ctl->loop_bound;
    const int cont = !ld_flag(&ctl->phase_done) && n < bound && n < (unsigned int)ctl->max_iter + 2u &&
                     (cap == 0u || n < cap);
    cudaGraphSetConditional(h, cont ? 1u : 0u);
}

}  // namespace lgf
