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
#include "lgf_dft.cuh"

namespace lgf {

__device__ __forceinline__ int ld_flag(const int* p) { return *(const volatile int*)p; }

// ---------------------------------------------------------------- tiles and line passes

// Occupancy floor of the tiled FFT kernels, compiled for line lengths up to
// LMAX: FP32 kernels (bound by memory latency) keep two blocks of 256 threads per
// SM, three when every line is at most 32 long; FP64 kernels (bound by the FP64
// pipe, which a few warps keep busy) may use every register.
template <typename T, int LMAX> constexpr int kTileMinBlocks = sizeof(T) == 4 ? (LMAX <= 32 ? 3 : 2) : (LMAX <= 32 ? 3 : 1);
// FP64 tiles run at most 128 threads per block (a 32-point line per thread needs
// ~160 registers; three such blocks per SM keep 12 warps on the FP64 pipe)
template <typename T> constexpr int kTileMaxThreads = sizeof(T) == 8 ? 128 : 256;

// Shared-memory tiles.  The xy-plane tile holds the four fields of one plane as
// [f][y][x] with row stride Lx + 1 (odd, so that the rows of consecutive lanes
// start in different banks) and field stride Ly (Lx + 1).  The z,t pencil tile
// of xw x-columns holds [t][kz][xi] with row stride rs = Lz xw, padded by xw when
// xw is narrower than one shared-memory wavefront (then consecutive t fall in
// different banks), followed by the pencil's multipliers [kt][kz][xi] (FP64) or
// the tables they are computed from (FP32).
__host__ __device__ inline int plane_rsx(const Lat& d) { return d.L[0] + 1; }
__host__ __device__ inline int plane_fs(const Lat& d) { return d.L[1] * (d.L[0] + 1); }
__host__ __device__ inline size_t plane_smem_bytes(const Lat& d, size_t elem) { return 4 * (size_t)plane_fs(d) * elem; }
__host__ __device__ inline int pencil_rs(const Lat& d, int xw, size_t elem)
{
    return (xw * (int)elem < 128 ? d.L[2] + 1 : d.L[2]) * xw;
}
// the pencil tile and, after it, FP64: the pencil's multipliers (xw Lz Lt
// doubles); FP32: the four tables of 4 sin^2(pi k / L) the multipliers are
// computed from
__host__ __device__ inline size_t pencil_smem_bytes(const Lat& d, int xw, size_t elem)
{
    const size_t tile = (size_t)d.L[3] * pencil_rs(d, xw, elem) * elem;
    if (elem == 8) return tile + (size_t)(d.L[0] + d.L[1] + d.L[2] + d.L[3]) * sizeof(float);
    return tile + (size_t)xw * d.L[2] * d.L[3] * sizeof(double);
}

// dst[i] = src(i) for i < n over the block, K loads in flight per thread before
// their stores (a load-then-store loop would wait out one memory latency per value)
template <int K, typename V, typename SRC, typename DST>
__device__ __forceinline__ void block_copy(int n, SRC src, DST dst)
{
    const int nt = blockDim.x;
    for (int i0 = threadIdx.x; i0 < n; i0 += K * nt) {
        V v[K];
#pragma unroll
        for (int u = 0; u < K; u++) {
            const int i = i0 + u * nt;
            if (i < n) v[u] = src(i);
        }
#pragma unroll
        for (int u = 0; u < K; u++) {
            const int i = i0 + u * nt;
            if (i < n) dst(i, v[u]);
        }
    }
}

// Transform nlines lines of length L (forward, or inverse when INV): each line
// is read through ld(line, position) and written through st(line, position,
// value), positions 0..L-1 along the line in natural order (time in, frequency
// out for the forward transform; the reverse for the inverse).  The lanes of a
// line (pass_lanes(L) of them) work together, so every thread of the block
// calls this with the same nlines; lines are dealt out a warp at a time.
// NL > 0 sets the lanes per line (default: pass_lanes).
template <typename T, int L, bool INV, int NL = 0, typename LD, typename ST>
__device__ __forceinline__ void lines_pass(int nlines, LD ld, ST st)
{
    constexpr int Tl = NL > 0 ? NL : pass_lanes<T>(L), R = L / Tl, W = 32 / Tl;
    const int lane = (int)threadIdx.x & 31, tau = lane / W, w = lane - tau * W;
    const int step = ((int)blockDim.x >> 5) * W;
    for (int l0 = ((int)threadIdx.x >> 5) * W; l0 < nlines; l0 += step) {
        const int l = l0 + w;
        const bool ok = l < nlines;
        const int lc = ok ? l : l0;
        cx<T> v[R];
#pragma unroll
        for (int j = 0; j < R; j++)
            v[j] = ld(lc, INV ? line_pos_k<T, L, Tl>(tau, j) : line_pos_x<T, L, Tl>(tau, j));
        if constexpr (INV) line_inv<T, L, Tl>(v, tau);
        else line_fwd<T, L, Tl>(v, tau);
        if (ok) {
#pragma unroll
            for (int j = 0; j < R; j++)
                st(l, INV ? line_pos_x<T, L, Tl>(tau, j) : line_pos_k<T, L, Tl>(tau, j), v[j]);
        }
    }
}

// Forward transform, a real multiplier per frequency m(line, k), inverse
// transform, in one pass over the lines (natural order in and out).
template <typename T, int L, typename LD, typename MUL, typename ST>
__device__ __forceinline__ void lines_accel(int nlines, LD ld, MUL mul, ST st)
{
    constexpr int Tl = line_lanes<T>(L), R = L / Tl, W = 32 / Tl;
    const int lane = (int)threadIdx.x & 31, tau = lane / W, w = lane - tau * W;
    const int step = ((int)blockDim.x >> 5) * W;
    for (int l0 = ((int)threadIdx.x >> 5) * W; l0 < nlines; l0 += step) {
        const int l = l0 + w;
        const bool ok = l < nlines;
        const int lc = ok ? l : l0;
        cx<T> v[R];
#pragma unroll
        for (int j = 0; j < R; j++) v[j] = ld(lc, line_pos_x<T, L>(tau, j));
        line_fwd<T, L>(v, tau);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const T m = mul(lc, line_pos_k<T, L>(tau, r));
            v[r].re *= m;
            v[r].im *= m;
        }
        line_inv<T, L>(v, tau);
        if (ok) {
#pragma unroll
            for (int j = 0; j < R; j++) st(l, line_pos_x<T, L>(tau, j), v[j]);
        }
    }
}

// The x-lines (rows) of the four fields of a plane tile, in place.
template <typename T, bool INV, int LMAX>
__device__ __forceinline__ void tile_x_lines(const Lat& d, vec2_t<T>* sm)
{
    const int Ly = d.L[1], rsx = plane_rsx(d), fs = plane_fs(d);
    with_length<LMAX>(d.L[0], [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        auto row = [&](int l) {
            const int f = (int)fdiv((unsigned)l, d.dLy), y = l - f * Ly;
            return sm + f * fs + y * rsx;
        };
        lines_pass<T, L, INV>(
            4 * Ly, [&](int l, int e) { return ldv<T>(row(l) + e); },
            [&](int l, int e, cx<T> v) { st<T>(row(l) + e, v); });
    });
}

// The y-lines (columns) of the four fields of a plane: loaded from src (the
// tile, or the plane's fields in global memory, [f][y][x] with field stride
// src_fs and row stride src_rs), transformed, stored to dst likewise.
template <typename T, bool INV, int LMAX>
__device__ __forceinline__ void plane_y_lines(const Lat& d, const vec2_t<T>* src, int src_fs, int src_rs,
                                              vec2_t<T>* dst, int dst_fs, int dst_rs)
{
    // offsets stay 32-bit: four fields of V sites, V < 2^31 / 24
    const int Lx = d.L[0];
    with_length<LMAX>(d.L[1], [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        lines_pass<T, L, INV>(
            4 * Lx,
            [&](int l, int e) {
                const int f = (int)fdiv((unsigned)l, d.dLx), x = l - f * Lx;
                return ldv<T>(src + (f * src_fs + e * src_rs + x));
            },
            [&](int l, int e, cx<T> v) {
                const int f = (int)fdiv((unsigned)l, d.dLx), x = l - f * Lx;
                st<T>(dst + (f * dst_fs + e * dst_rs + x), v);
            });
    });
}

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

// per-site sum of |Delta_ij|^2 of the packed Delta, in T
template <typename T> __device__ __forceinline__ T theta_site(const cx<T>* D)
{
    const T p = D[3].re, q = D[3].im, pq = p + q;
    return (T)2 * (norm2(D[0]) + norm2(D[1]) + norm2(D[2])) + p * p + q * q + pq * pq;
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

// Delta rounded to the precision of the transform (TF): FP64 -> FP32 on the
// integer pipe (d2f_int, round to nearest even)
template <typename TF> __device__ __forceinline__ cx<TF> to_tf(cx<double> v)
{
    if constexpr (sizeof(TF) == 8) return v;
    else return mk<float>(d2f_int(v.re), d2f_int(v.im));
}

// One block per xy-plane.  Delta(x) = sum_mu ah_mu(x - mu) - ah_mu(x) (packed
// fields), theta and F reduced in FP64; with FFT, the forward transform along x
// (rows of the plane tile) and y (columns, stored straight to Fd), else Delta
// itself to Fd.  Shared memory: the plane tile (FFT only).  TF: precision of the
// transform and of Fd (FP64 links with TF = float: Delta, theta and F from the
// FP64 parts, the transform in FP32).
template <typename T, bool FFT, int LMAX, typename TF = T>
__global__ void __launch_bounds__(kTileMaxThreads<T>, kTileMinBlocks<T, LMAX>) k_delta(Lat d, const vec2_t<T>* __restrict__ AH, const T* __restrict__ Fs,
                                               vec2_t<TF>* __restrict__ Fd, double* __restrict__ partials, Ctl* ctl,
                                               double2* hist)
{
    static_assert(sizeof(T) == sizeof(TF) || sizeof(T) == 8, "FP32 links take FP32 transforms");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<TF>* sm = reinterpret_cast<vec2_t<TF>*>(smem_raw);
    if (ld_flag(&ctl->phase_done)) return;
    const int P = d.P, V = d.V, Lx = d.L[0];
    const int plane = blockIdx.x;
    const int s0 = plane * P;
    const int z = plane % d.L[2], t = plane / d.L[2];
    const int rsx = plane_rsx(d), fs = plane_fs(d);
    double th = 0.0, fsum = 0.0;
    if constexpr (sizeof(T) == 4) {
        // FP32: two sites (x, x+1) per thread, every part loaded as a pair of sites
        // in one 16-byte load (x even; the neighbours along y, z, t are pairs too,
        // and along x the pair's first neighbour is x - 1, its second x itself)
        const float4* AH4 = reinterpret_cast<const float4*>(AH);
        const int V2 = V / 2;
#pragma unroll 1
        for (int xy = 2 * threadIdx.x; xy < P; xy += 2 * blockDim.x) {
            const int s = s0 + xy;
            const int y = (int)fdiv((unsigned)xy, d.dLx), x = xy - y * Lx;
            const int c[4] = {x, y, z, t};
            int sb[4];
#pragma unroll
            for (int mu = 1; mu < 4; mu++) sb[mu] = site_shift(d, s, c[mu], mu, -1);
            sb[0] = site_shift(d, s, x, 0, -1);
            const float2 fs2 = __ldg(reinterpret_cast<const float2*>(Fs) + s / 2);
            fsum += (double)fs2.x + (double)fs2.y;
            cx<float> D0[4], D1[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                // site x: ah_x(x-1) - ah_x(x); site x+1: ah_x(x) - ah_x(x+1)
                const float4 b = __ldg(AH4 + (size_t)k * V2 + s / 2);
                const float2 a = __ldg(AH + (size_t)k * V + sb[0]);
                D0[k] = mk<float>(a.x - b.x, a.y - b.y);
                D1[k] = mk<float>(b.x - b.z, b.y - b.w);
            }
#pragma unroll
            for (int mu = 1; mu < 4; mu++)
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float4 a = __ldg(AH4 + (size_t)(mu * 4 + k) * V2 + sb[mu] / 2);
                    const float4 b = __ldg(AH4 + (size_t)(mu * 4 + k) * V2 + s / 2);
                    D0[k] = D0[k] + mk<float>(a.x - b.x, a.y - b.y);
                    D1[k] = D1[k] + mk<float>(a.z - b.z, a.w - b.w);
                }
            th += (double)theta_site(D0) + (double)theta_site(D1);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (FFT) {
                    st<float>(reinterpret_cast<float2*>(sm) + k * fs + y * rsx + x, D0[k]);
                    st<float>(reinterpret_cast<float2*>(sm) + k * fs + y * rsx + x + 1, D1[k]);
                } else {
                    st<float>(reinterpret_cast<float2*>(Fd) + (size_t)k * V + s, D0[k]);
                    st<float>(reinterpret_cast<float2*>(Fd) + (size_t)k * V + s + 1, D1[k]);
                }
            }
        }
    } else {
#pragma unroll 2
    for (int xy = threadIdx.x; xy < P; xy += blockDim.x) {
        const int s = s0 + xy;
        const int y = (int)fdiv((unsigned)xy, d.dLx), x = xy - y * Lx;
        const int c[4] = {x, y, z, t};
        int sb[4];
#pragma unroll
        for (int mu = 0; mu < 4; mu++) sb[mu] = site_shift(d, s, c[mu], mu, -1);
        // every load of the site issued before the arithmetic
        cx<T> a[16], b[16];
#pragma unroll
        for (int mu = 0; mu < 4; mu++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                a[4 * mu + k] = ld<T>(AH + (size_t)(mu * 4 + k) * V + sb[mu]);
                b[4 * mu + k] = ld<T>(AH + (size_t)(mu * 4 + k) * V + s);
            }
        fsum += (double)__ldg(Fs + s);
        cx<T> D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            D[k] = a[k] - b[k];
#pragma unroll
            for (int mu = 1; mu < 4; mu++) D[k] = D[k] + a[4 * mu + k] - b[4 * mu + k];
        }
        // per-site sum of |Delta_ij|^2 in the kernel's precision, accumulated over
        // sites in FP64
        th += (double)theta_site(D);
        if (FFT) {
#pragma unroll
            for (int k = 0; k < 4; k++) st<TF>(sm + k * fs + y * rsx + x, to_tf<TF>(D[k]));
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) st<TF>(Fd + (size_t)k * V + s, to_tf<TF>(D[k]));
        }
    }
    }
    reduce_theta_F(th, fsum, partials, ctl, hist, V);
    if (FFT) {
        __syncthreads();
        tile_x_lines<TF, false, LMAX>(d, sm);
        __syncthreads();
        plane_y_lines<TF, false, LMAX>(d, sm, fs, rsx, Fd + s0, V, Lx);
    }
}

// ---------------------------------------------------------------- k_zt

// One block per (x-chunk of xw columns, y, field); the fields arrive transformed
// along x and y, so x and y are the momenta kx, ky.  The accelerator
// p2max/(p2(k) V), zero mode removed, comes in FP64 from mult (the table of
// multipliers, site-indexed by momentum), staged in shared memory for the
// pencil; in FP32 it is computed from the FP32 tables s2f of 4 sin^2(pi k/L)
// (with alpha/2 folded in, see k_xyinv_g).  z-lines are read from Fd into
// registers and transformed forward, stored to the pencil tile [t][kz][xi]; each
// t-line is transformed forward, multiplied by the accelerator and transformed
// back; the z-lines are transformed back and written to Fd.
template <typename T, int LMAX>
__global__ void __launch_bounds__(kTileMaxThreads<T>, kTileMinBlocks<T, LMAX>) k_zt(Lat d, int xw, vec2_t<T>* __restrict__ Fd,
                                                                     const Ctl* ctl, const double* __restrict__ mult,
                                                                     const float* __restrict__ s2f, float p2max_v)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    if (ld_flag(&ctl->phase_done)) return;
    const int Lx = d.L[0], Ly = d.L[1], Lz = d.L[2], Lt = d.L[3];
    const int P = d.P;  // offsets stay 32-bit (V < 2^31 / 24)
    const int rs = pencil_rs(d, xw, sizeof(vec2_t<T>));
    const int xs = __ffs(xw) - 1;  // xw is a power of two
    const int x0 = (int)blockIdx.x * xw, ky = (int)blockIdx.y;
    const int c0 = x0 + Lx * ky;  // (kx0, ky)
    vec2_t<T>* g = Fd + (size_t)blockIdx.z * d.V + c0;
    // FP64: the pencil's multipliers [kt][kz][xi]; FP32: the tables sx, sy, sz, st
    double* m64 = reinterpret_cast<double*>(sm + Lt * rs);
    float* t32 = reinterpret_cast<float*>(sm + Lt * rs);
    float hc = 0.f;
    if constexpr (sizeof(T) == 8) {
        const double* mrow = mult + c0;
        block_copy<8, double>(
            xw * Lz * Lt,
            [&](int i) {
                const int zt = i >> xs, xi = i & (xw - 1);
                return __ldg(mrow + (xi + P * zt));
            },
            [&](int i, double v) { m64[i] = v; });
    } else {
        // alpha/2 p2max / V (p2max_v = p2max / V); the g builder of the FP32 phase
        // then takes the field as alpha/2 Delta~
        hc = 0.5f * (float)ctl->alpha * p2max_v;
        block_copy<4, float>(Lx + Ly + Lz + Lt, [&](int i) { return __ldg(s2f + i); },
                             [&](int i, float v) { t32[i] = v; });
    }
    // z forward: lines (xi, t)
    with_length<LMAX>(Lz, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        lines_pass<T, L, false>(
            xw * Lt,
            [&](int l, int e) {
                const int tt = l >> xs, xi = l & (xw - 1);
                return ldv<T>(g + (xi + P * (e + L * tt)));
            },
            [&](int l, int e, cx<T> v) {
                const int tt = l >> xs, xi = l & (xw - 1);
                st<T>(sm + tt * rs + e * xw + xi, v);
            });
    });
    __syncthreads();
    // t forward, accelerator, t inverse: lines (xi, kz)
    with_length<LMAX>(Lt, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        lines_accel<T, L>(
            xw * Lz, [&](int l, int e) { return ldv<T>(sm + e * rs + l); },
            [&](int l, int k) -> T {
                if constexpr (sizeof(T) == 8) {
                    return m64[l + xw * Lz * k];
                } else {
                    const int kz = l >> xs, xi = l & (xw - 1);
                    const float p2 = t32[x0 + xi] + t32[Lx + ky] + t32[Lx + Ly + kz] + t32[Lx + Ly + Lz + k];
                    return p2 > 0.f ? __fdividef(hc, p2) : 0.f;
                }
            },
            [&](int l, int e, cx<T> v) { st<T>(sm + e * rs + l, v); });
    });
    __syncthreads();
    // z inverse: lines (xi, t), back to Fd
    with_length<LMAX>(Lz, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        lines_pass<T, L, true>(
            xw * Lt,
            [&](int l, int e) {
                const int tt = l >> xs, xi = l & (xw - 1);
                return ldv<T>(sm + tt * rs + e * xw + xi);
            },
            [&](int l, int e, cx<T> v) {
                const int tt = l >> xs, xi = l & (xw - 1);
                st<T>(g + (xi + P * (e + L * tt)), v);
            });
    });
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

// One xy-plane by one block: inverse transform along y (columns read from Fd)
// and x (rows of the plane tile sm), then g = reunit(1 + alpha/2 Delta~) by row
// Gram-Schmidt in FP64 whatever T is; g stored as TG.
template <typename T, typename TG, int LMAX>
__device__ __forceinline__ void xyinv_g_plane(const Lat& d, const vec2_t<T>* __restrict__ Fd,
                                              vec2_t<TG>* __restrict__ g, const Ctl* ctl, int plane, vec2_t<T>* sm)
{
    const int P = d.P, V = d.V, Lx = d.L[0];
    const int s0 = plane * P;
    const int rsx = plane_rsx(d), fs = plane_fs(d);
    plane_y_lines<T, true, LMAX>(d, Fd + s0, V, Lx, sm, fs, rsx);
    __syncthreads();
    tile_x_lines<T, true, LMAX>(d, sm);
    __syncthreads();
    for (int xy = threadIdx.x; xy < P; xy += blockDim.x) {
        const int y = (int)fdiv((unsigned)xy, d.dLx), x = xy - y * Lx;
        const int o = y * rsx + x;
        vec2_t<T> f0 = sm[o], f1 = sm[fs + o], f2 = sm[2 * fs + o], f3 = sm[3 * fs + o];
        // X = 1 + (alpha/2) Delta~ ; rows 0 and 1 (FP32 fields arrive already
        // multiplied by alpha/2, in the z,t kernel)
        cx<double> X[6];
        if constexpr (sizeof(T) == 4) {
            // conversions on the integer pipe (f2d_int, d2f_int below): a fifth
            // of this kernel's FP64-pipe work otherwise
            const double a0 = f2d_int(f0.x), a1 = f2d_int(f0.y);
            X[0] = mk<double>(1.0, f2d_int(f3.x));
            X[1] = mk<double>(a0, a1);
            X[2] = mk<double>(f2d_int(f1.x), f2d_int(f1.y));
            X[3] = mk<double>(-a0, a1);  // -conj(Delta01)
            X[4] = mk<double>(1.0, f2d_int(f3.y));
            X[5] = mk<double>(f2d_int(f2.x), f2d_int(f2.y));
        } else {
            const double h = 0.5 * ctl->alpha;
            X[0] = mk<double>(1.0, h * f3.x);
            X[1] = mk<double>(h * f0.x, h * f0.y);
            X[2] = mk<double>(h * f1.x, h * f1.y);
            X[3] = mk<double>(-h * f0.x, h * f0.y);  // -conj(Delta01)
            X[4] = mk<double>(1.0, h * f3.y);
            X[5] = mk<double>(h * f2.x, h * f2.y);
        }
        // Gram-Schmidt in FP64; row 2 = conj(r0 x r1) in the precision g is
        // stored in (for an FP32 g, from the rounded rows, so that the stored g
        // is unitary to FP32 rounding)
        cx<double> gm[6];
        gram_schmidt01(X, gm);
        cx<TG> gs[9];
        if constexpr (sizeof(TG) == 4) {
#pragma unroll
            for (int e = 0; e < 6; e++) gs[e] = mk<TG>(d2f_int(gm[e].re), d2f_int(gm[e].im));
        } else {
#pragma unroll
            for (int e = 0; e < 6; e++) gs[e] = mk<TG>((TG)gm[e].re, (TG)gm[e].im);
        }
        complete_row2(gs, gs + 6);
#pragma unroll
        for (int e = 0; e < 9; e++) st<TG>(g + (size_t)e * V + s0 + xy, gs[e]);
    }
}

// One block per xy-plane (xyinv_g_plane).
template <typename T, typename TG, int LMAX>
__global__ void __launch_bounds__(kTileMaxThreads<T>, kTileMinBlocks<T, LMAX>) k_xyinv_g(Lat d, const vec2_t<T>* __restrict__ Fd,
                                                 vec2_t<TG>* __restrict__ g, const Ctl* ctl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    if (ld_flag(&ctl->phase_done)) return;
    xyinv_g_plane<T, TG, LMAX>(d, Fd, g, ctl, blockIdx.x, sm);
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

// w = ga u gb^dag for full 3x3 ga, u, gb: rows 0,1 as two 2x3-by-3x3 products,
// row 2 rebuilt as conj(row0 x row1) (the 12-real form of the result)
template <typename T>
__device__ __forceinline__ void link_gug(const cx<T>* ga, const cx<T>* u, const cx<T>* gb, cx<T>* w)
{
    cx<T> A[6];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> acc = cmul(ga[3 * i], u[j]);
            acc = cmac(acc, ga[3 * i + 1], u[3 + j]);
            acc = cmac(acc, ga[3 * i + 2], u[6 + j]);
            A[3 * i + j] = acc;
        }
    // w_ij = sum_k A_ik conj(gb_jk)
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<T> acc = cmulc(A[3 * i], gb[3 * j]);
            acc = cmacc(acc, A[3 * i + 1], gb[3 * j + 1]);
            acc = cmacc(acc, A[3 * i + 2], gb[3 * j + 2]);
            w[3 * i + j] = acc;
        }
    complete_row2(w, w + 6);
}

// G(x) <- g(x) G(x), rows 0,1 stored (row 2 of G rebuilt on load)
template <typename T>
__device__ __forceinline__ void gauge_accumulate(vec2_t<T>* __restrict__ G, int V, int s, const cx<T>* gx)
{
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

// One thread per site.  G may be null (gauge not tracked).  Also writes the
// packed anti-Hermitian parts of the new links (AH) and their Re Tr per site
// (Fs) for the next Delta.
// The update of site s (see k_update); ldg(e, site) loads entry e of g at site.
template <typename T, typename LDG>
__device__ __forceinline__ void update_site(const Lat& d, vec2_t<T>* __restrict__ U, vec2_t<T>* __restrict__ G,
                                            LDG ldg, vec2_t<T>* __restrict__ AH, T* __restrict__ Fs, int s)
{
    const int V = d.V;
    int c[4];
    site_coords(d, s, c);
    cx<T> gx[9];
#pragma unroll
    for (int e = 0; e < 9; e++) gx[e] = ldg(e, s);
    T f = 0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<T> u[9], gn[9], w[9];
        load_link<T>(U, V, d.ne, mu, s, u);
        const int sn = site_shift(d, s, c[mu], mu, +1);
#pragma unroll
        for (int e = 0; e < 9; e++) gn[e] = ldg(e, sn);
        link_gug(gx, u, gn, w);
        store_link<T>(U, V, d.ne, mu, s, w);
        cx<T> a[4];
        ah_pack(w, a);
#pragma unroll
        for (int k = 0; k < 4; k++) st<T>(AH + (size_t)(mu * 4 + k) * V + s, a[k]);
        f += w[0].re + w[4].re + w[8].re;
    }
    Fs[s] = f;
    if (G != nullptr) gauge_accumulate<T>(G, V, s, gx);
}

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
    update_site<T>(d, U, G, [&](int e, int site) { return ld<T>(g + (size_t)e * V + site); }, AH, Fs, s);
}

// ---------------------------------------------------------------- g builder and update in one launch

// Work queue of the persistent g-and-update kernel over the xy-planes
// p = z + Lz t: items "build g of plane p" (inverse x,y transform and FP64
// Gram-Schmidt: the FP64 pipe) and "update the sites of plane p" (HBM).  The
// update of plane (z, t) reads g at (z, t), (z+1, t) and (z, t+1), so the queue
// holds the builds of t in [0, lag), then for each t < Lt - lag the builds of
// t + lag followed by the updates of t, then the updates of the last lag values
// of t: every update comes after the builds it reads, which blocks that were
// running took earlier, so waiting for them cannot deadlock; a lag of about the
// resident blocks over Lz keeps most builds finished before their updates are
// taken.
struct GuItem {
    int build, plane;
};
__host__ __device__ __forceinline__ GuItem gu_item(int i, int Lz, int Lt, int lag)
{
    const int nA = lag * Lz;
    if (i < nA) return GuItem{1, i};
    const int j = i - nA, nB = 2 * (Lt - lag) * Lz;
    if (j < nB) {
        const int t = j / (2 * Lz), r = j - t * 2 * Lz;
        return r < Lz ? GuItem{1, (t + lag) * Lz + r} : GuItem{0, t * Lz + (r - Lz)};
    }
    return GuItem{0, (Lt - lag) * Lz + (j - nB)};
}

// wait until *flag >= ep (another block's release); false after ~1 s of the
// global timer
__device__ __forceinline__ bool wait_flag_ge(const unsigned* flag, unsigned ep)
{
    if (*(const volatile unsigned*)flag >= ep) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        for (int k = 0; k < 32; k++)
            if (*(const volatile unsigned*)flag >= ep) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
        __nanosleep(64);
    }
}

// The FP32 phase's g builder and update in one persistent launch (queue above).
// Sync words (per context, zeroed once): [0] next item, [1] blocks finished,
// [2] launches completed (the epoch), [3] unused, then one word per plane: the
// epoch of the launch that last built the plane's g.  A build item ends with a
// block barrier and a release of its flag by thread 0; an update item's thread 0
// waits for the three flags it reads and the block then reads g through L2 (it
// was written in this launch).  A wait that runs out sets Ctl::fault; the last
// block to finish then stops the loop.  The last block also counts the
// iteration, resets the queue and advances the epoch.
template <typename T, int LMAX>
__global__ void __launch_bounds__(kTileMaxThreads<T>, kTileMinBlocks<T, LMAX>) k_gu(
    Lat d, const vec2_t<T>* __restrict__ Fd, vec2_t<T>* __restrict__ g, vec2_t<T>* __restrict__ U,
    vec2_t<T>* __restrict__ G, vec2_t<T>* __restrict__ AH, T* __restrict__ Fs, Ctl* ctl, unsigned* sync, int lag)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* sm = reinterpret_cast<vec2_t<T>*>(smem_raw);
    __shared__ int s_item;
    if (ld_flag(&ctl->phase_done)) return;
    const int Lz = d.L[2], Lt = d.L[3], P = d.P, V = d.V;
    const int nitems = 2 * d.nplanes;
    unsigned* flags = sync + 4;
    const unsigned ep = *(const volatile unsigned*)(sync + 2) + 1u;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(sync, 1u);
        __syncthreads();
        const int i = s_item;
        __syncthreads();
        if (i >= nitems) break;
        const GuItem it = gu_item(i, Lz, Lt, lag);
        if (it.build) {
            xyinv_g_plane<T, T, LMAX>(d, Fd, g, ctl, it.plane, sm);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(flags + it.plane, ep);
            }
        } else {
            if (threadIdx.x == 0) {
                const int z = it.plane % Lz, t = it.plane / Lz;
                const int dep[3] = {it.plane, (z + 1 == Lz ? 0 : z + 1) + Lz * t, z + Lz * (t + 1 == Lt ? 0 : t + 1)};
                bool ok = true;
#pragma unroll
                for (int k = 0; k < 3; k++) ok = wait_flag_ge(flags + dep[k], ep) && ok;
                if (!ok) atomicExch(&ctl->fault, 1);
                __threadfence();
            }
            __syncthreads();
            const int s0 = it.plane * P;
            for (int xy = threadIdx.x; xy < P; xy += blockDim.x)
                update_site<T>(
                    d, U, G,
                    [&](int e, int site) {
                        const vec2_t<T> v = __ldcg(g + (size_t)e * V + site);
                        return mk<T>(v.x, v.y);
                    },
                    AH, Fs, s0 + xy);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned tk = atomicAdd(sync + 1, 1u);
        if (tk == gridDim.x - 1) {
            ctl->iter += 1;
            if (ctl->phase == 0) ctl->iter_phase0 += 1;
            if (ld_flag(&ctl->fault)) {
                ctl->phase_done = 1;
                ctl->done = 1;
            }
            sync[0] = 0u;
            sync[1] = 0u;
            __threadfence();
            atomicExch(sync + 2, ep);
        }
    }
}

// ---------------------------------------------------------------- fused update and Delta

// The update fused with the Delta stencil (the form of the FP32 phase, where
// recomputing a neighbour's link costs less than moving its anti-Hermitian part
// through memory).  One thread per site x:
//   U'_mu(x) = g(x) U_mu(x) g^dag(x+mu), stored to Uout, and G(x) <- g(x) G(x);
//   the links entering x, U'_mu(x-mu) = g(x-mu) U_mu(x-mu) g^dag(x), recomputed
//   from Uin for their anti-Hermitian parts only;
//   Delta(x) = sum_mu ah(U'_mu(x-mu)) - ah(U'_mu(x)) stored to Fd (packed, in
//   space), theta and F of the new links reduced in FP64, the loop state updated.
// Uin and Uout are different buffers: a thread reads its neighbours' old links,
// which their own threads replace in the same launch.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_update_delta(
    Lat d, const vec2_t<T>* __restrict__ Uin, vec2_t<T>* __restrict__ Uout, vec2_t<T>* __restrict__ G,
    const vec2_t<T>* __restrict__ g, Ctl* ctl, vec2_t<T>* __restrict__ Fd, double* __restrict__ partials,
    double2* hist)
{
    if (ld_flag(&ctl->phase_done)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->iter += 1;
        if (ctl->phase == 0) ctl->iter_phase0 += 1;
    }
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double th = 0.0, fsum = 0.0;
    if (s < V) {
        int c[4];
        site_coords(d, s, c);
        cx<T> gx[9];
        load_g<T>(g, V, s, gx);
        cx<T> D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) D[k] = mk<T>(0, 0);
        T f = 0;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            cx<T> u[9], gn[9], w[9], a[4];
            // the link leaving x
            load_link<T>(Uin, V, d.ne, mu, s, u);
            load_g<T>(g, V, site_shift(d, s, c[mu], mu, +1), gn);
            link_gug(gx, u, gn, w);
            store_link<T>(Uout, V, d.ne, mu, s, w);
            ah_pack(w, a);
#pragma unroll
            for (int k = 0; k < 4; k++) D[k] = D[k] - a[k];
            f += w[0].re + w[4].re + w[8].re;
            // the link entering x from x - mu
            const int sb = site_shift(d, s, c[mu], mu, -1);
            load_link<T>(Uin, V, d.ne, mu, sb, u);
            load_g<T>(g, V, sb, gn);
            link_gug(gn, u, gx, w);
            ah_pack(w, a);
#pragma unroll
            for (int k = 0; k < 4; k++) D[k] = D[k] + a[k];
        }
        if (G != nullptr) gauge_accumulate<T>(G, V, s, gx);
#pragma unroll
        for (int k = 0; k < 4; k++) st<T>(Fd + (size_t)k * V + s, D[k]);
        th = (double)theta_site(D);
        fsum = (double)f;
    }
    reduce_theta_F(th, fsum, partials, ctl, hist, V);
}

// Delta, theta and F of the stored links themselves (no update): the start of
// the FP32 phase and, when `every` > 0, the iterations on which the FP32 links
// were rebuilt from the FP64 input (the refresh).  Delta in space to Fd.
template <typename T>
__global__ void __launch_bounds__(256) k_delta_links(Lat d, const vec2_t<T>* __restrict__ U,
                                                     vec2_t<T>* __restrict__ Fd, double* __restrict__ partials,
                                                     Ctl* ctl, double2* hist, int every)
{
    if (ld_flag(&ctl->phase_done)) return;
    if (every > 0 && !(ctl->phase == 0 && ctl->iter > 0 && ctl->iter % every == 0)) return;
    const int V = d.V;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double th = 0.0, fsum = 0.0;
    if (s < V) {
        int c[4];
        site_coords(d, s, c);
        cx<T> D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) D[k] = mk<T>(0, 0);
        T f = 0;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            cx<T> u[9], a[4];
            load_link<T>(U, V, d.ne, mu, s, u);
            ah_pack(u, a);
#pragma unroll
            for (int k = 0; k < 4; k++) D[k] = D[k] - a[k];
            f += u[0].re + u[4].re + u[8].re;
            load_link<T>(U, V, d.ne, mu, site_shift(d, s, c[mu], mu, -1), u);
            ah_pack(u, a);
#pragma unroll
            for (int k = 0; k < 4; k++) D[k] = D[k] + a[k];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) st<T>(Fd + (size_t)k * V + s, D[k]);
        th = (double)theta_site(D);
        fsum = (double)f;
    }
    reduce_theta_F(th, fsum, partials, ctl, hist, V);
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
