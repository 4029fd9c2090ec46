// The z,t transform of the FP32 phase with whole lines in registers, for lattices
// with Lz = Lt = N in {8, 16, 32}: the same computation as k_zt (forward FFT along
// z and t of the four packed Delta fields, the accelerator p2max/(p2(k) V) with the
// zero mode removed, inverse FFT along t and z), organised for an FP32 phase whose
// fields sit in L2: one thread transforms one line of N points held in registers
// (radix 2, twiddles as compile-time constants), so a launch has four barriers instead of one
// per Stockham stage and no twiddle loads.
//
// One block per (x-chunk of XW columns, y, field), XW * N threads.  The tile holds
// value (z or kz, t or kt, xi) at t * RS + z * XW + xi (RS pads a row of N * XW
// values so that consecutive t fall in different shared-memory banks), the
// multipliers of the block's momenta in the same order (row stride N * XW).
//   load: the pencil and its multipliers, coalesced, into the tiles.
//   A: thread (xi, t) transforms its z-line forward (decimation in frequency,
//      bit-reversed order out) and stores each frequency in its natural row.
//   B: thread (xi, kz) transforms its t-line forward, multiplies by the
//      accelerator, transforms back (decimation in time from bit-reversed order,
//      natural order out) and stores it in place.
//   C: thread (xi, t) transforms its z-line back (read in bit-reversed order).
//   store: the pencil, coalesced.
// Both directions are unnormalised; the 1/V is in the multiplier table.
#pragma once
#include "lgf_common.cuh"
#include "lgf_fft.cuh"

namespace lgf {

// cos(pi m / 16), m = 0..8
__host__ __device__ constexpr float cos_pi16(int m)
{
    return m == 0   ? 1.0f
           : m == 1 ? 0.98078528040323044913f
           : m == 2 ? 0.92387953251128675613f
           : m == 3 ? 0.83146961230254523708f
           : m == 4 ? 0.70710678118654752440f
           : m == 5 ? 0.55557023301960222474f
           : m == 6 ? 0.38268343236508977173f
           : m == 7 ? 0.19509032201612826785f
                    : 0.0f;
}

// w_N^e = exp(-2 pi i e / N) for 0 <= e < N/2 (conjugated for the inverse), as
// a power of w_32: cos and sin of pi e' / 16 with e' = e * 32 / N < 16.
template <int N, bool INV> __device__ __forceinline__ cx<float> root(int e)
{
    const int m = e * (32 / N);
    const float c = m <= 8 ? cos_pi16(m) : -cos_pi16(16 - m);
    const float s = m <= 8 ? cos_pi16(8 - m) : cos_pi16(m - 8);  // sin(pi m / 16)
    return mk(c, INV ? s : -s);
}

__host__ __device__ constexpr int bitrev(int k, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((k >> b) & 1) << (bits - 1 - b);
    return r;
}

__host__ __device__ constexpr int log2i(int n) { return n <= 1 ? 0 : 1 + log2i(n / 2); }

// radix-2 decimation in frequency: natural order in, v[k] = X[bitrev(k)] out
template <int N, bool INV> __device__ __forceinline__ void lines_dif(cx<float>* v)
{
#pragma unroll
    for (int span = N / 2; span >= 1; span >>= 1)
#pragma unroll
        for (int b = 0; b < N; b += 2 * span)
#pragma unroll
            for (int j = 0; j < span; j++) {
                const cx<float> a = v[b + j], c = v[b + j + span];
                const cx<float> d = a - c;
                v[b + j] = a + c;
                v[b + j + span] = j == 0 ? d : cmul(d, root<N, INV>(j * (N / (2 * span))));
            }
}

// radix-2 decimation in time: v[k] = x[bitrev(k)] in, natural order out
template <int N, bool INV> __device__ __forceinline__ void lines_dit(cx<float>* v)
{
#pragma unroll
    for (int span = 1; span < N; span <<= 1)
#pragma unroll
        for (int b = 0; b < N; b += 2 * span)
#pragma unroll
            for (int j = 0; j < span; j++) {
                const cx<float> a = v[b + j];
                const cx<float> c = j == 0 ? v[b + j + span] : cmul(v[b + j + span], root<N, INV>(j * (N / (2 * span))));
                v[b + j] = a + c;
                v[b + j + span] = a - c;
            }
}

constexpr int kZtLinesMaxThreads = 512;

// row stride of the data tile: N * XW values, plus XW when a row spans whole
// 128-byte bank windows and a group of XW values does not
template <int N, int XW> __host__ __device__ constexpr int zt_lines_rs()
{
    return N * XW + (((N * XW * 8) % 128 == 0 && XW * 8 < 128) ? XW : 0);
}

template <int N, int XW> __host__ __device__ constexpr size_t zt_lines_smem_bytes()
{
    return (size_t)N * zt_lines_rs<N, XW>() * sizeof(float2) + (size_t)N * N * XW * sizeof(float);
}

template <int N, int XW>
__global__ void __launch_bounds__(N * XW) k_zt_lines(Lat d, float2* __restrict__ Fd, const Ctl* ctl,
                                                     const float* __restrict__ mult)
{
    constexpr int B = log2i(N), RS = zt_lines_rs<N, XW>(), NT = N * XW, NV = N * N * XW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tile = reinterpret_cast<float2*>(smem_raw);
    float* mt = reinterpret_cast<float*>(tile + N * RS);
    if (ld_flag(&ctl->phase_done)) return;
    const size_t P = (size_t)d.P;
    const size_t c0 = (size_t)blockIdx.x * XW + (size_t)d.L[0] * blockIdx.y;  // (kx0, ky) of the block
    float2* base = Fd + (size_t)blockIdx.z * d.V + c0;
    const float* mbase = mult + c0;
    // value i = xi + XW (z + N t) of the pencil
#pragma unroll 4
    for (int i = threadIdx.x; i < NV; i += NT) {
        const int zt = i / XW, xi = i - zt * XW, t = zt / N;
        tile[i + t * (RS - N * XW)] = base[xi + P * zt];
        mt[i] = __ldg(mbase + xi + P * zt);
    }
    __syncthreads();
    const int xi = (int)threadIdx.x % XW, r = (int)threadIdx.x / XW;
    cx<float> v[N];
    // A: the z-line at t = r; frequency bitrev(k) back to row bitrev(k)
    {
        float2* line = tile + r * RS + xi;
#pragma unroll
        for (int z = 0; z < N; z++) v[z] = ldv<float>(line + z * XW);
        lines_dif<N, false>(v);
#pragma unroll
        for (int k = 0; k < N; k++) st<float>(line + bitrev(k, B) * XW, v[k]);
    }
    __syncthreads();
    // B: the t-line of row kz = r
    {
        float2* line = tile + r * XW + xi;
        const float* mline = mt + r * XW + xi;
#pragma unroll
        for (int t = 0; t < N; t++) v[t] = ldv<float>(line + t * RS);
        lines_dif<N, false>(v);
#pragma unroll
        for (int k = 0; k < N; k++) v[k] = v[k] * mline[bitrev(k, B) * NT];  // kt = bitrev(k)
        lines_dit<N, true>(v);
#pragma unroll
        for (int t = 0; t < N; t++) st<float>(line + t * RS, v[t]);
    }
    __syncthreads();
    // C: the z-line at t = r, read in bit-reversed order
    {
        float2* line = tile + r * RS + xi;
#pragma unroll
        for (int k = 0; k < N; k++) v[k] = ldv<float>(line + bitrev(k, B) * XW);
        lines_dit<N, true>(v);
#pragma unroll
        for (int z = 0; z < N; z++) st<float>(line + z * XW, v[z]);
    }
    __syncthreads();
#pragma unroll 4
    for (int i = threadIdx.x; i < NV; i += NT) {
        const int zt = i / XW, xi = i - zt * XW, t = zt / N;
        base[xi + P * zt] = tile[i + t * (RS - N * XW)];
    }
}

// the line kernels take Lz = Lt = N in {8, 16, 32} and pencils of XW in {4, 8, 16}
// columns (N * XW <= 512 threads); returns N, else 0
inline int zt_lines_n(const Lat& d, int xw)
{
    const int n = d.L[2];
    if (d.L[3] != n || (n != 8 && n != 16 && n != 32)) return 0;
    if ((xw != 4 && xw != 8 && xw != 16) || xw * n > kZtLinesMaxThreads) return 0;
    return n;
}

template <int N, int XW> inline void launch_zt_lines_nx(dim3 grid, cudaStream_t s, const Lat& d, float2* Fd,
                                                        const Ctl* ctl, const float* mult)
{
    k_zt_lines<N, XW><<<grid, N * XW, zt_lines_smem_bytes<N, XW>(), s>>>(d, Fd, ctl, mult);
}

template <int N> inline void launch_zt_lines_n(int xw, dim3 grid, cudaStream_t s, const Lat& d, float2* Fd,
                                               const Ctl* ctl, const float* mult)
{
    if (xw == 4) launch_zt_lines_nx<N, 4>(grid, s, d, Fd, ctl, mult);
    else if (xw == 8) launch_zt_lines_nx<N, 8>(grid, s, d, Fd, ctl, mult);
    else launch_zt_lines_nx<N, 16>(grid, s, d, Fd, ctl, mult);
}

// launch for a lattice that zt_lines_n accepts: grid (Lx / xw, Ly, 4)
inline void launch_zt_lines(int n, int xw, cudaStream_t s, const Lat& d, float2* Fd, const Ctl* ctl, const float* mult)
{
    const dim3 grid((unsigned)(d.L[0] / xw), (unsigned)d.L[1], 4);
    if (n == 8) launch_zt_lines_n<8>(xw, grid, s, d, Fd, ctl, mult);
    else if (n == 16) launch_zt_lines_n<16>(xw, grid, s, d, Fd, ctl, mult);
    else launch_zt_lines_n<32>(xw, grid, s, d, Fd, ctl, mult);
}

}  // namespace lgf
