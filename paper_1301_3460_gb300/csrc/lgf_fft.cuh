// Batched 1D complex FFTs on lines held in shared memory (Stockham auto-sort,
// mixed radix 2/3/4/8, out of place: each stage reads one shared-memory buffer
// and writes the other, so a thread holds one butterfly at a time).  Used along x and y inside the xy-plane kernels and
// along z and t inside the zt-pencil kernel: a 4D transform of the Delta
// colour fields is the product of the four 1D transforms (the forward and
// inverse transforms of the Fourier-accelerated step).
//
// Stage s with radix R and NS = product of the earlier radices maps, for the
// butterfly j < L/R with k = j mod NS,
//   v_r = x[j + r L/R] * w_L^{r k L/(NS R)},  v = DFT_R(v),
//   y[(j div NS) NS R + k + r NS] = v_r,
// which leaves the transform in natural order after the last stage.
#pragma once
#include "lgf_common.cuh"

namespace lgf {

// ---------------------------------------------------------------- index helpers

// Division by a run-time constant d as a multiply-high and a shift (exact for
// numerators below 2^31): s = ceil(log2 d), m = floor(2^32 (2^s - d)/d) + 1,
// n / d = (umulhi(n, m) + n) >> s.
struct FDiv {
    unsigned m, s;
};
inline FDiv make_fdiv(unsigned d)
{
    unsigned s = 0;
    while ((1u << s) < d) s++;
    const unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1ull;
    return FDiv{(unsigned)m, s};
}
__device__ __forceinline__ unsigned fdq(unsigned n, FDiv f) { return (__umulhi(n, f.m) + n) >> f.s; }

// element e of line l sits at buf[(l / A) * B + (l % A) * C + e * ES]
struct LineMap {
    FDiv fA;
    unsigned A, B, C, ES;
    __device__ __forceinline__ unsigned base(unsigned l) const
    {
        const unsigned q = fdq(l, fA);
        return q * B + (l - q * A) * C;
    }
};
inline LineMap make_linemap(unsigned A, unsigned B, unsigned C, unsigned ES)
{
    return LineMap{make_fdiv(A), A, B, C, ES};
}

// Stages of one transform length: radix R, NS = product of the earlier radices,
// tws = L / (NS R) (twiddle table stride), with the divisions by NB = L/R and
// NS precomputed.
struct AxisPlan {
    int L, nst;
    int R[4], NS[4], tws[4];
    FDiv fNB[4], fNS[4];
};

// batch of lines: count and the divider for it
struct Lines {
    unsigned n;
    FDiv fn;
};
inline Lines make_lines(unsigned n) { return Lines{n, make_fdiv(n)}; }

// ---------------------------------------------------------------- small DFTs

// The transform direction is a run-time value so that one inlined copy of the
// code serves both: i*z is multiplied by sgn = -1 (forward, exp(-i..)) or +1
// (inverse), applied as a sign-bit flip (an integer operation).
__device__ __forceinline__ double flip(double x, unsigned m)
{
    return __hiloint2double(__double2hiint(x) ^ (int)m, __double2loint(x));
}
__device__ __forceinline__ float flip(float x, unsigned m) { return __uint_as_float(__float_as_uint(x) ^ m); }

// sgn * i * z with sgn = -1 when m is the sign mask, +1 when m = 0
template <typename T> __device__ __forceinline__ cx<T> mul_si(cx<T> z, unsigned m)
{
    return mk<T>(flip(z.im, m ^ 0x80000000u), flip(z.re, m));
}

template <typename T> __device__ __forceinline__ void dft2(cx<T>* v, unsigned)
{
    cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <typename T> __device__ __forceinline__ void dft3(cx<T>* v, unsigned m)
{
    const T h = (T)0.86602540378443864676372317075294;  // sqrt(3)/2
    cx<T> t1 = v[1] + v[2];
    cx<T> t2 = v[1] - v[2];
    cx<T> c = v[0] - t1 * (T)0.5;
    v[0] = v[0] + t1;
    // forward: y1 = c - i q, y2 = c + i q, q = h t2 (inverse: i -> -i)
    cx<T> iq = mul_si(t2 * h, m);
    v[1] = c + iq;
    v[2] = c - iq;
}

template <typename T> __device__ __forceinline__ void dft4v(cx<T>& a, cx<T>& b, cx<T>& c, cx<T>& d, unsigned m)
{
    cx<T> t0 = a + c, t1 = a - c, t2 = b + d, t3 = b - d;
    cx<T> it3 = mul_si(t3, m);  // forward: -i t3
    a = t0 + t2;
    c = t0 - t2;
    b = t1 + it3;
    d = t1 - it3;
}

template <typename T> __device__ __forceinline__ void dft4(cx<T>* v, unsigned m) { dft4v<T>(v[0], v[1], v[2], v[3], m); }

template <typename T> __device__ __forceinline__ void dft8(cx<T>* v, unsigned m)
{
    const T r = (T)0.70710678118654752440084436210485;  // 1/sqrt(2)
    cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4v<T>(e0, e1, e2, e3, m);
    dft4v<T>(o0, o1, o2, o3, m);
    // o_k *= w8^k, w8 = exp(sgn i pi/4) = (1 + sgn i)/sqrt(2)
    o1 = (o1 + mul_si(o1, m)) * r;
    o2 = mul_si(o2, m);
    o3 = (mul_si(o3, m) - o3) * r;  // w8^3 = (-1 + sgn i)/sqrt(2)
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + o1;
    v[5] = e1 - o1;
    v[2] = e2 + o2;
    v[6] = e2 - o2;
    v[3] = e3 + o3;
    v[7] = e3 - o3;
}

template <typename T, int R> __device__ __forceinline__ void dftR(cx<T>* v, unsigned m)
{
    if constexpr (R == 2) dft2<T>(v, m);
    else if constexpr (R == 3) dft3<T>(v, m);
    else if constexpr (R == 4) dft4<T>(v, m);
    else dft8<T>(v, m);
}

// ---------------------------------------------------------------- plans

__host__ __device__ constexpr bool fft_length_supported(int L)
{
    return L == 4 || L == 6 || L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64 ||
           L == 96 || L == 128;
}

// radices of each supported length, first stage first
inline AxisPlan make_axis_plan(int L)
{
    AxisPlan p{};
    p.L = L;
    int r[4] = {0, 0, 0, 0};
    switch (L) {
    case 4: r[0] = 4; break;
    case 6: r[0] = 2; r[1] = 3; break;
    case 8: r[0] = 8; break;
    case 12: r[0] = 4; r[1] = 3; break;
    case 16: r[0] = 4; r[1] = 4; break;
    case 24: r[0] = 8; r[1] = 3; break;
    case 32: r[0] = 8; r[1] = 4; break;
    case 48: r[0] = 4; r[1] = 4; r[2] = 3; break;
    case 64: r[0] = 8; r[1] = 8; break;
    case 96: r[0] = 8; r[1] = 4; r[2] = 3; break;
    case 128: r[0] = 8; r[1] = 4; r[2] = 4; break;
    default: break;
    }
    int ns = 1;
    for (int i = 0; i < 4 && r[i]; i++) {
        p.R[i] = r[i];
        p.NS[i] = ns;
        p.tws[i] = L / (ns * r[i]);
        p.fNB[i] = make_fdiv((unsigned)(L / r[i]));
        p.fNS[i] = make_fdiv((unsigned)ns);
        ns *= r[i];
        p.nst = i + 1;
    }
    return p;
}

// ---------------------------------------------------------------- one stage

// Direction masks: kFwd for exp(-2 pi i ...), kInv for exp(+2 pi i ...).
constexpr unsigned kFwd = 0x80000000u, kInv = 0u;

// One Stockham stage over all lines, src -> dst (same layout).  All threads of
// the block take part; a barrier ends the stage.  line_fast: consecutive items
// walk consecutive lines (for lines interleaved in memory); otherwise
// consecutive items walk the butterflies of one line.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const vec2_t<T>* src, vec2_t<T>* dst, const Lines ln, int line_fast,
                                          const LineMap& mp, const AxisPlan& ap, int st,
                                          const vec2_t<T>* __restrict__ tw, unsigned dir)
{
    const unsigned NB = (unsigned)(ap.L / R);
    const unsigned NS = (unsigned)ap.NS[st];
    const unsigned tws = (unsigned)ap.tws[st];
    const FDiv fNB = ap.fNB[st], fNS = ap.fNS[st];
    const unsigned nitems = ln.n * NB;
    for (unsigned it = threadIdx.x; it < nitems; it += blockDim.x) {
        unsigned l, j;
        if (line_fast) {
            j = fdq(it, ln.fn);
            l = it - j * ln.n;
        } else {
            l = fdq(it, fNB);
            j = it - l * NB;
        }
        const unsigned b = mp.base(l);
        const unsigned q = fdq(j, fNS);
        const unsigned k = j - q * NS;
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            vec2_t<T> x = src[b + (j + r * NB) * mp.ES];
            v[r] = mk<T>(x.x, x.y);
        }
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                cx<T> w = ld<T>(tw + r * k * tws);  // exp(-2 pi i ...)
                w.im = flip(w.im, dir ^ kFwd);      // conjugate for the inverse
                v[r] = cmul(v[r], w);
            }
        }
        dftR<T, R>(v, dir);
        const unsigned d0 = q * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) {
            vec2_t<T> x;
            x.x = v[r].re;
            x.y = v[r].im;
            dst[b + (d0 + r * NS) * mp.ES] = x;
        }
    }
    __syncthreads();
}

// Transform the lines held in a (layout mp) using b as the other buffer, in
// direction dir with tw[m] = exp(-2 pi i m / L); unnormalised both ways.
// Returns the buffer (a or b) that holds the result.
template <typename T>
__device__ __forceinline__ vec2_t<T>* fft_lines(const AxisPlan& ap, vec2_t<T>* a, vec2_t<T>* b, const Lines ln,
                                                int line_fast, const LineMap& mp, const vec2_t<T>* __restrict__ tw,
                                                unsigned dir)
{
#pragma unroll 1
    for (int st = 0; st < ap.nst; st++) {
        const int R = ap.R[st];
        if (R == 8) fft_stage<T, 8>(a, b, ln, line_fast, mp, ap, st, tw, dir);
        else if (R == 4) fft_stage<T, 4>(a, b, ln, line_fast, mp, ap, st, tw, dir);
        else if (R == 3) fft_stage<T, 3>(a, b, ln, line_fast, mp, ap, st, tw, dir);
        else fft_stage<T, 2>(a, b, ln, line_fast, mp, ap, st, tw, dir);
        vec2_t<T>* t = a;
        a = b;
        b = t;
    }
    return a;
}

// Plans and line maps of the two plane-tiled transforms: the xy-plane ([f][y][x],
// chunks of nfc fields) and the zt-pencil ([t][z][xi] of xw columns).
struct XyFft {
    AxisPlan px, py;
    LineMap mx, my;   // x-lines (rows) and y-lines (columns) of a chunk
    Lines lx, ly;     // nfc*Ly rows, nfc*Lx columns
    int nfc;
};
struct ZtFft {
    AxisPlan pz, pt;
    LineMap mz, mt;
    Lines lz, lt;     // xw*Lt z-lines, xw*Lz t-lines
    int xw;
    int rs;           // row stride (values) of the [t][z][xi] tile: Lz*xw, maybe padded
};

// Plans and maps of the [t][z][xi] pencil tile of xw x-columns.  Consecutive
// threads take the z-lines of consecutive (xi, t): groups of xw values one row
// apart.  When a row spans whole 128-byte bank windows and a group does not,
// the row is padded by xw values so that the groups of consecutive t fall in
// different banks instead of the same ones.
inline ZtFft make_zt_fft(int Lz, int Lt, int xw, size_t elem)
{
    ZtFft Z{};
    Z.pz = make_axis_plan(Lz);
    Z.pt = make_axis_plan(Lt);
    unsigned rs = (unsigned)(Lz * xw);
    if ((rs * elem) % 128 == 0 && xw * elem < 128) rs += (unsigned)xw;
    Z.mz = make_linemap((unsigned)xw, rs, 1, (unsigned)xw);
    Z.mt = make_linemap(1u << 30, 0, 1, rs);
    Z.lz = make_lines((unsigned)(xw * Lt));
    Z.lt = make_lines((unsigned)(xw * Lz));
    Z.xw = xw;
    Z.rs = (int)rs;
    return Z;
}

// shared memory of the two pencil buffers
inline size_t zt_tile_bytes(const ZtFft& Z, int Lt, size_t elem) { return (size_t)2 * Lt * Z.rs * elem; }

// The four Delta fields of one xy-plane in a = [f][y][x] (4 P values), with
// scratch b of nfc P values: transform along x then y, chunk by chunk; the
// result is left in a.
template <typename T>
__device__ __forceinline__ void fft_xy_fields(const XyFft& F, int P, vec2_t<T>* a, vec2_t<T>* b,
                                              const vec2_t<T>* __restrict__ twx, const vec2_t<T>* __restrict__ twy,
                                              unsigned dir)
{
#pragma unroll 1
    for (int f0 = 0; f0 < 4; f0 += F.nfc) {
        vec2_t<T>* home = a + f0 * P;
        vec2_t<T>* r = fft_lines<T>(F.px, home, b, F.lx, 0, F.mx, twx, dir);
        r = fft_lines<T>(F.py, r, r == home ? b : home, F.ly, 1, F.my, twy, dir);
        if (r != home) {
            for (int i = threadIdx.x; i < F.nfc * P; i += blockDim.x) home[i] = r[i];
            __syncthreads();
        }
    }
}

}  // namespace lgf
