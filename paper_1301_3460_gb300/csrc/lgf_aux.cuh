// Kernels around the iteration: conversion between the caller's
// [..][3][3] complex128 arrays and the library's 12-real planes, the SU(3)
// check of input links, stand-alone stage kernels, and the precision switch of
// the mixed mode (FP32 phase -> FP64 phase).
#pragma once
#include "lgf_kernels.cuh"

namespace lgf {

__device__ __forceinline__ double dmax_nan(double a, double b)
{
    // NaN counts as larger than anything
    if (!(a == a)) return a;
    if (!(b == b)) return b;
    return a > b ? a : b;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v)
{
    if (!(v <= 1e300)) v = 1e300;  // NaN and inf compare as huge
    // non-negative doubles order like their bit patterns
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Interleaved [4][V][3][3] complex128 -> rows 0,1 planes of T; optional SU(3)
// check of the full input matrix: err[0] = max |U U^dag - 1|, err[1] = max |det U - 1|,
// err[2] = max error of the round trip through the 8-real form (ne = 4).
template <typename T>
static __global__ void k_pack_links(int V, int ne, const double* __restrict__ in, vec2_t<T>* __restrict__ U,
                             unsigned long long* err, int validate)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;  // link index mu*V + s
    // squared errors, their square root taken once after the maximum (the square
    // root is monotone and correctly rounded, so this is the maximum of the errors)
    double e_unit = 0.0, e_det = 0.0, e_form = 0.0;
    if (idx < 4L * V) {
        const int mu = (int)(idx / V), s = (int)(idx - (long)mu * V);
        const double* p = in + idx * 18;  // 8-byte loads: the caller's array need not be 16-byte aligned
        cx<double> m[9];
#pragma unroll
        for (int e = 0; e < 9; e++) m[e] = mk<double>(p[2 * e], p[2 * e + 1]);
        if (ne == 4) {
            // 8-real form; the check below also covers its round trip (the form
            // cannot hold links with |u00| = 1, such as the unit matrix)
            cx<T> w[9];
#pragma unroll
            for (int e = 0; e < 9; e++) w[e] = mk<T>((T)m[e].re, (T)m[e].im);
            store_link<T>(U, V, 4, mu, s, w);
            if (validate) {
                cx<T> r[9];
                rebuild8<T>(w[1], w[2], w[3], atan2(w[0].im, w[0].re), atan2(w[6].im, w[6].re), r);
#pragma unroll
                for (int e = 0; e < 9; e++) e_form = dmax_nan(e_form, (double)norm2(r[e] - w[e]));
            }
        } else {
#pragma unroll
            for (int e = 0; e < 6; e++) {
                vec2_t<T> v;
                v.x = (T)m[e].re;
                v.y = (T)m[e].im;
                U[(size_t)(mu * ne + e) * V + s] = v;
            }
        }
        if (ne == 9) {
            // row 2 stored as the rebuild from rows 0,1, as a 12-real load would give it
            cx<T> r[9];
#pragma unroll
            for (int e = 0; e < 6; e++) r[e] = mk<T>((T)m[e].re, (T)m[e].im);
            complete_row2(r, r + 6);
#pragma unroll
            for (int e = 6; e < 9; e++) st<T>(U + (size_t)(mu * 9 + e) * V + s, r[e]);
        }
        if (validate) {
            // U U^dag is Hermitian: its entries (i, j) with i <= j (the entry (j, i)
            // is their conjugate up to the last rounding of one product)
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = i; j < 3; j++) {
                    cx<double> acc = cmulc(m[3 * i], m[3 * j]);
                    acc = cmacc(acc, m[3 * i + 1], m[3 * j + 1]);
                    acc = cmacc(acc, m[3 * i + 2], m[3 * j + 2]);
                    if (i == j) acc.re -= 1.0;
                    e_unit = dmax_nan(e_unit, norm2(acc));
                }
            cx<double> r2[3];
            complete_row2(m, r2);  // conj of the cofactor row: det = sum_j m2j conj(r2_j)
            cx<double> det = cmulc(m[6], r2[0]);
            det = cmacc(det, m[7], r2[1]);
            det = cmacc(det, m[8], r2[2]);
            det.re -= 1.0;
            e_det = norm2(det);
            if (!(e_det == e_det)) e_det = 1e300;
        }
    }
    if (validate) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e_unit = dmax_nan(e_unit, __shfl_down_sync(0xffffffffu, e_unit, o));
            e_det = dmax_nan(e_det, __shfl_down_sync(0xffffffffu, e_det, o));
            e_form = dmax_nan(e_form, __shfl_down_sync(0xffffffffu, e_form, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_nonneg(err, sqrt(e_unit));
            atomic_max_nonneg(err + 1, sqrt(e_det));
            atomic_max_nonneg(err + 2, sqrt(e_form));
        }
    }
}

// [nmat][ne][V] planes -> interleaved [nmat][V][3][3] complex128 (row 2 rebuilt or read)
template <typename T>
static __global__ void k_unpack_su3(int V, int nmat, int ne, const vec2_t<T>* __restrict__ U, double* __restrict__ out)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nmat * V) return;
    const int mu = (int)(idx / V), s = (int)(idx - (long)mu * V);
    cx<T> m[9];
    load_link<T>(U, V, ne, mu, s, m);
    double* p = out + idx * 18;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        p[2 * e] = (double)m[e].re;
        p[2 * e + 1] = (double)m[e].im;
    }
}

template <typename T> __global__ void k_identity_rows(int V, vec2_t<T>* __restrict__ G)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int e = 0; e < 6; e++) {
        vec2_t<T> v;
        v.x = (e == 0 || e == 4) ? (T)1 : (T)0;
        v.y = (T)0;
        G[(size_t)e * V + s] = v;
    }
}

// [V][3][3] traceless anti-Hermitian complex128 -> the four packed fields
static __global__ void k_pack_delta(int V, const double* __restrict__ in, double2* __restrict__ Fd)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const double* p = in + (size_t)s * 18;
    Fd[s] = make_double2(p[2], p[3]);                 // Delta01
    Fd[(size_t)V + s] = make_double2(p[4], p[5]);     // Delta02
    Fd[(size_t)2 * V + s] = make_double2(p[10], p[11]);  // Delta12
    Fd[(size_t)3 * V + s] = make_double2(p[1], p[9]);    // Im Delta00 + i Im Delta11
}

// the four packed fields -> [V][3][3] traceless anti-Hermitian complex128
static __global__ void k_unpack_delta(int V, const double2* __restrict__ Fd, double* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const double2 d01 = Fd[s], d02 = Fd[(size_t)V + s], d12 = Fd[(size_t)2 * V + s], ab = Fd[(size_t)3 * V + s];
    double* p = out + (size_t)s * 18;
    const double m[18] = {0.0, ab.x, d01.x, d01.y, d02.x, d02.y, -d01.x, d01.y, 0.0, ab.y,
                          d12.x, d12.y, -d02.x, d02.y, -d12.x, d12.y, 0.0, -(ab.x + ab.y)};
#pragma unroll
    for (int e = 0; e < 18; e++) p[e] = m[e];
}

// n complex values from FP64 to FP32 and back, times a real scale (the FP32
// stage entry points: their inputs and outputs are FP64)
static __global__ void k_planes_to32(long n, const double2* __restrict__ in, float2* __restrict__ out, double scale)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = in[i];
    out[i] = make_float2((float)(v.x * scale), (float)(v.y * scale));
}
static __global__ void k_planes_to64(long n, const float2* __restrict__ in, double2* __restrict__ out, double scale)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 v = in[i];
    out[i] = make_double2((double)v.x * scale, (double)v.y * scale);
}

// [9][V] planes of full matrices -> [V][3][3] complex128
static __global__ void k_unpack_full(int V, const double2* __restrict__ g, double* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double* p = out + (size_t)s * 18;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        const double2 v = g[(size_t)e * V + s];
        p[2 * e] = v.x;
        p[2 * e + 1] = v.y;
    }
}

// plane-wise FFT along x and y of the four fields, in place on Fd (stand-alone
// stage; one block per xy-plane, the plane tile in shared memory)
template <typename T, bool INV, int LMAX>
__global__ void __launch_bounds__(kTileMaxThreads<T>, kTileMinBlocks<T, LMAX>) k_xy_fft(Lat d, vec2_t<T>* __restrict__ Fd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    const int P = d.P, V = d.V, Lx = d.L[0], s0 = blockIdx.x * P;
    const int rsx = plane_rsx(d), fs = plane_fs(d);
    vec2_t<T>* base = Fd + s0;
    if (INV) {
        plane_y_lines<T, true, LMAX>(d, base, V, Lx, sm, fs, rsx);
        __syncthreads();
        tile_x_lines<T, true, LMAX>(d, sm);
        __syncthreads();
        block_copy<4, vec2_t<T>>(
            4 * P,
            [&](int i) {
                const int f = (int)fdiv((unsigned)i, d.dP), xy = i - f * P, y = (int)fdiv((unsigned)xy, d.dLx), x = xy - y * Lx;
                return sm[f * fs + y * rsx + x];
            },
            [&](int i, vec2_t<T> v) {
                const int f = (int)fdiv((unsigned)i, d.dP), xy = i - f * P;
                base[(size_t)f * V + xy] = v;
            });
    } else {
        block_copy<8, vec2_t<T>>(
            4 * P,
            [&](int i) {
                const int f = (int)fdiv((unsigned)i, d.dP), xy = i - f * P;
                return base[(size_t)f * V + xy];
            },
            [&](int i, vec2_t<T> v) {
                const int f = (int)fdiv((unsigned)i, d.dP), xy = i - f * P, y = (int)fdiv((unsigned)xy, d.dLx), x = xy - y * Lx;
                sm[f * fs + y * rsx + x] = v;
            });
        __syncthreads();
        tile_x_lines<T, false, LMAX>(d, sm);
        __syncthreads();
        plane_y_lines<T, false, LMAX>(d, sm, fs, rsx, base, V, Lx);
    }
}

// ---------------------------------------------------------------- mixed mode

// start of the FP32 phase: FP32 copy (rows 0,1) of the current FP64 links
// (layout [mu][ne][V]), G32 = 1
static __global__ void k_mixed_prep(int V, int ne, const double2* __restrict__ U64, float2* __restrict__ U32,
                             float2* __restrict__ G32, const Ctl* ctl)
{
    if (ld_flag(&ctl->done)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<double> u[9];
        load_link<double>(U64, V, ne, mu, s, u);
#pragma unroll
        for (int e = 0; e < 6; e++) U32[(size_t)(mu * 6 + e) * V + s] = make_float2((float)u[e].re, (float)u[e].im);
    }
#pragma unroll
    for (int e = 0; e < 6; e++) G32[(size_t)e * V + s] = make_float2((e == 0 || e == 4) ? 1.f : 0.f, 0.f);
}

// end of the FP32 phase: Gs = reunit(G32) in FP64, stored as full 3x3 planes.
// Runs also when the FP32 phase used up max_iter, so that the stored links keep
// its progress; only a NaN skips it.
static __global__ void k_switch_gs(int V, const float2* __restrict__ G32, double2* __restrict__ Gs, const Ctl* ctl)
{
    if (ld_flag(&ctl->nan_seen)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    cx<double> X[6], g[9];
#pragma unroll
    for (int e = 0; e < 6; e++) {
        const float2 v = G32[(size_t)e * V + s];
        X[e] = mk<double>((double)v.x, (double)v.y);
    }
    reunit_rows(X, g);
#pragma unroll
    for (int e = 0; e < 9; e++) Gs[(size_t)e * V + s] = make_double2(g[e].re, g[e].im);
}

// U_mu(x) <- Gs(x) U_mu(x) Gs^dag(x+mu) and G(x) <- Gs(x) G(x), FP64, in place
static __global__ void __launch_bounds__(256) k_project(Lat d, double2* __restrict__ U, double2* __restrict__ G,
                                                const double2* __restrict__ Gs, const Ctl* ctl)
{
    if (ld_flag(&ctl->nan_seen)) return;
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    cx<double> gx[9];
    load_g<double>(Gs, V, s, gx);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<double> u[9];
        load_link<double>(U, V, d.ne, mu, s, u);
        cx<double> A[6];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<double> acc = cmul(gx[3 * i], u[j]);
                acc = cmac(acc, gx[3 * i + 1], u[3 + j]);
                acc = cmac(acc, gx[3 * i + 2], u[6 + j]);
                A[3 * i + j] = acc;
            }
        cx<double> gn[9];
        load_g<double>(Gs, V, site_shift(d, s, c[mu], mu, +1), gn);
        cx<double> w[9];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<double> acc = cmulc(A[3 * i], gn[3 * j]);
                acc = cmacc(acc, A[3 * i + 1], gn[3 * j + 1]);
                acc = cmacc(acc, A[3 * i + 2], gn[3 * j + 2]);
                w[3 * i + j] = acc;
            }
        complete_row2(w, w + 6);
        store_link<double>(U, V, d.ne, mu, s, w);
    }
    if (G != nullptr) {
        cx<double> Gm[9];
#pragma unroll
        for (int e = 0; e < 6; e++) Gm[e] = ldv<double>(G + (size_t)e * V + s);
        complete_row2(Gm, Gm + 6);
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<double> acc = cmul(gx[3 * i], Gm[j]);
                acc = cmac(acc, gx[3 * i + 1], Gm[3 + j]);
                acc = cmac(acc, gx[3 * i + 2], Gm[6 + j]);
                st<double>(G + (size_t)(3 * i + j) * V + s, acc);
            }
    }
}

// ---------------------------------------------------------------- FP32-phase refresh
//
// The FP32 links drift off the input's gauge orbit by FP32 rounding at every
// update, and the drift grows with the iteration count; at the switch the FP64
// links are rebuilt on the orbit from G, so the FP64 finish has to remove
// whatever the FP32 links had drifted.  Every `every` FP32 updates the links are
// therefore rebuilt from the input and the (re-orthonormalised) G:
//   G(x) <- reunit(G(x)),  U32_mu(x) <- G(x) U_in_mu(x) G^dag(x+mu)
// (with the packed anti-Hermitian parts and Re Tr of the new links when AH and
// Fs are given; the fused FP32 iteration recomputes Delta from the links).

__device__ __forceinline__ bool refresh_due(const Ctl* ctl, int every)
{
    if (ld_flag(&ctl->phase_done) || ctl->phase != 0) return false;
    return every > 0 && ctl->iter > 0 && ctl->iter % every == 0;
}

// rows 0,1 of G32 re-orthonormalised (Gram-Schmidt in FP64)
static __global__ void k_refresh_g(int V, float2* __restrict__ G32, const Ctl* ctl, int every)
{
    if (!refresh_due(ctl, every)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    cx<double> X[6], g[9];
#pragma unroll
    for (int e = 0; e < 6; e++) {
        const float2 v = G32[(size_t)e * V + s];
        X[e] = mk<double>((double)v.x, (double)v.y);
    }
    reunit_rows(X, g);
#pragma unroll
    for (int e = 0; e < 6; e++) G32[(size_t)e * V + s] = make_float2((float)g[e].re, (float)g[e].im);
}

// U32 = G U_in G^dag(x+mu) in FP32 from the FP64 input links (ne64 stored entries)
static __global__ void __launch_bounds__(256) k_refresh_u(Lat d, int ne64, const double2* __restrict__ U64,
                                                          const float2* __restrict__ G32, float2* __restrict__ U32,
                                                          float2* __restrict__ AH, float* __restrict__ Fs,
                                                          const Ctl* ctl, int every)
{
    if (!refresh_due(ctl, every)) return;
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    cx<float> gx[9];
#pragma unroll
    for (int e = 0; e < 6; e++) gx[e] = ld<float>(G32 + (size_t)e * V + s);
    complete_row2(gx, gx + 6);
    float f = 0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<float> u[9];
        {
            cx<double> ud[9];
            load_link<double>(U64, V, ne64, mu, s, ud);
#pragma unroll
            for (int e = 0; e < 6; e++) u[e] = mk<float>((float)ud[e].re, (float)ud[e].im);
        }
        complete_row2(u, u + 6);
        cx<float> A[6];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<float> acc = cmul(gx[3 * i], u[j]);
                acc = cmac(acc, gx[3 * i + 1], u[3 + j]);
                acc = cmac(acc, gx[3 * i + 2], u[6 + j]);
                A[3 * i + j] = acc;
            }
        const int sn = site_shift(d, s, c[mu], mu, +1);
        cx<float> gn[9];
#pragma unroll
        for (int e = 0; e < 6; e++) gn[e] = ld<float>(G32 + (size_t)e * V + sn);
        complete_row2(gn, gn + 6);
        cx<float> w[9];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                cx<float> acc = cmulc(A[3 * i], gn[3 * j]);
                acc = cmacc(acc, A[3 * i + 1], gn[3 * j + 1]);
                acc = cmacc(acc, A[3 * i + 2], gn[3 * j + 2]);
                w[3 * i + j] = acc;
                st<float>(U32 + (size_t)(mu * 6 + 3 * i + j) * V + s, acc);
            }
        complete_row2(w, w + 6);
        if (AH != nullptr) {
            cx<float> a[4];
            ah_pack(w, a);
#pragma unroll
            for (int k = 0; k < 4; k++) st<float>(AH + (size_t)(mu * 4 + k) * V + s, a[k]);
        }
        f += w[0].re + w[4].re + w[8].re;
    }
    if (Fs != nullptr) Fs[s] = f;
}

// hand over from the FP32 phase to the FP64 phase
static __global__ void k_phase_switch(Ctl* ctl)
{
    if (ld_flag(&ctl->done)) return;
    ctl->phase = 1;
    ctl->tol = ctl->tol_final;
    ctl->phase_done = 0;
    ctl->body_runs = 0u;
}

}  // namespace lgf
