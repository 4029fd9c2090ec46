// Register-resident discrete Fourier transforms for the 4D transform of the
// packed Delta fields (the forward and inverse FFT of the Fourier-accelerated
// step, described in the paper's introduction and GPU section).
//
// Codelets.  dft<T, N, INV>(v) transforms N complex values held in a register
// array, natural order in and out (the lengths 2, 3, 4, 6, 8, 12, 16, 24, 32,
// 48 and 96 appear):
//   N = 2^k * 3 (k >= 1): prime-factor (Good-Thomas) split into coprime factors
//                         2^k and 3, which needs no twiddle factors;
//   N = 2^k >= 8:         radix-2 decimation in time over two half-length
//                         codelets, each twiddled butterfly written as the
//                         six fused multiply-adds of the tangent form
//                         a +- w b = a +- w_r (b_r - (w_i/w_r) b_i, b_i + (w_i/w_r) b_r)
//                         (factoring the larger of w_r, w_i);
//   N = 2, 3, 4:          written out.
// Every index and root of unity is a compile-time constant, so the
// permutations are register renaming and trivial roots (1, -1, +-i) cost no
// arithmetic.  Forward is exp(-2 pi i n k / N), inverse exp(+2 pi i n k / N),
// both unnormalised.
//
// Lines.  A line of length L is held by T = line_lanes(L) lanes of one warp,
// R = L / T values per lane (one to eight lanes by length and precision).
// Lane tau (0 <= tau < T) holds x[tau + T j], j < R.  Forward:
//   1. the R-point codelet over j in each lane: Y_tau[r];
//   2. Y_tau[r] *= w_L^(tau r) (compile-time roots picked by lane);
//   3. the T-point transform across the lanes for each r, radix-2 decimation
//      in frequency by warp shuffles (roots 1 and -i applied by exchanging and
//      negating components; the eighth roots of T = 8 picked by lane).
// Lane tau then holds X[r + R bitrev_T(tau)].  The inverse takes that layout,
// runs the three steps backwards with conjugate roots and returns
// L x[tau + T j] in the input layout.
#pragma once
#include <type_traits>

#include "lgf_common.cuh"

namespace lgf {

// ---------------------------------------------------------------- constants

// cos(2 pi m / 384) for 0 <= m <= 96 (evaluated to 21 digits)
__host__ __device__ constexpr double cos384q(int m)
{
    return m == 0 ? 1.0
           : m == 1 ? 0.999866137909561782863
           : m == 2 ? 0.99946458747636564443
           : m == 3 ? 0.998795456205172392715
           : m == 4 ? 0.997858923238603506738
           : m == 5 ? 0.996655239309180324932
           : m == 6 ? 0.995184726672196886245
           : m == 7 ? 0.993447779019444395514
           : m == 8 ? 0.991444861373810411145
           : m == 9 ? 0.989176509964780973452
           : m == 10 ? 0.986643332084879004747
           : m == 11 ? 0.983846005927077416087
           : m == 12 ? 0.980785280403230449126
           : m == 13 ? 0.977461974943571863388
           : m == 14 ? 0.97387697927733364815
           : m == 15 ? 0.970031253194543992604
           : m == 16 ? 0.96592582628906828675
           : m == 17 ? 0.961561797682961947145
           : m == 18 ? 0.956940335732208864936
           : m == 19 ? 0.9520626777139242571
           : m == 20 ? 0.946930129495105664256
           : m == 21 ? 0.941544065183020778413
           : m == 22 ? 0.935905926757325700292
           : m == 23 ? 0.930017223684012117057
           : m == 24 ? 0.923879532511286756128
           : m == 25 ? 0.917494496447491307924
           : m == 26 ? 0.910863824921175818573
           : m == 27 ? 0.903989293123443331586
           : m == 28 ? 0.896872741532688303894
           : m == 29 ? 0.889516075421856035272
           : m == 30 ? 0.881921264348355029713
           : m == 31 ? 0.874090341626758851545
           : m == 32 ? 0.866025403784438646764
           : m == 33 ? 0.857728610000272069902
           : m == 34 ? 0.849202181526578887649
           : m == 35 ? 0.840448401094438021017
           : m == 36 ? 0.831469612302545237079
           : m == 37 ? 0.822268218989775107838
           : m == 38 ? 0.812846684591615216579
           : m == 39 ? 0.803207531480644909807
           : m == 40 ? 0.79335334029123516458
           : m == 41 ? 0.783286749228650365398
           : m == 42 ? 0.773010453362736960811
           : m == 43 ? 0.762527203906388096373
           : m == 44 ? 0.751839807478977396408
           : m == 45 ? 0.740951125354959091176
           : m == 46 ? 0.72986407269783565735
           : m == 47 ? 0.718581617779698057196
           : m == 48 ? 0.707106781186547524401
           : m == 49 ? 0.695442635009611651124
           : m == 50 ? 0.683592302022871280513
           : m == 51 ? 0.671558954847018400625
           : m == 52 ? 0.659345815100068868425
           : m == 53 ? 0.646956152534857365398
           : m == 54 ? 0.634393284163645498215
           : m == 55 ? 0.621660573370077408038
           : m == 56 ? 0.608761429008720639416
           : m == 57 ? 0.595699304492433343467
           : m == 58 ? 0.582477696867802149197
           : m == 59 ? 0.569100145878898230611
           : m == 60 ? 0.555570233019602224743
           : m == 61 ? 0.541891580574751716151
           : m == 62 ? 0.528067850650367995873
           : m == 63 ? 0.514102744193221726594
           : m == 64 ? 0.5
           : m == 65 ? 0.485763393716340056269
           : m == 66 ? 0.471396736825997648556
           : m == 67 ? 0.456903875630420676564
           : m == 68 ? 0.442288690219001281995
           : m == 69 ? 0.427555093430282094321
           : m == 70 ? 0.412707029804394737048
           : m == 71 ? 0.397748474527011052047
           : m == 72 ? 0.382683432365089771728
           : m == 73 ? 0.367515936594703565414
           : m == 74 ? 0.352250047921233506532
           : m == 75 ? 0.336889853392220050689
           : m == 76 ? 0.321439465303161580701
           : m == 77 ? 0.305903020096553462763
           : m == 78 ? 0.290284677254462367636
           : m == 79 ? 0.27458861818493234148
           : m == 80 ? 0.258819045102520762349
           : m == 81 ? 0.242980179903263889948
           : m == 82 ? 0.227076263034373207586
           : m == 83 ? 0.211111552358965165924
           : m == 84 ? 0.195090322016128267848
           : m == 85 ? 0.17901686127663268204
           : m == 86 ? 0.162895473394588739481
           : m == 87 ? 0.146730474455361751659
           : m == 88 ? 0.130526192220051591548
           : m == 89 ? 0.114286964966846398117
           : m == 90 ? 0.0980171403295606019942
           : m == 91 ? 0.0817210741336682237477
           : m == 92 ? 0.0654031292301430668153
           : m == 93 ? 0.049067674327418014255
           : m == 94 ? 0.0327190828217761420637
           : m == 95 ? 0.016361731626486781643
           : 0.0;
}

// cos and sin of 2 pi m / 384 for any integer m, by the quadrant symmetries
// (every line length and codelet length divides 384)
__host__ __device__ constexpr double cos384(int m)
{
    m %= 384;
    if (m < 0) m += 384;
    if (m > 192) m = 384 - m;
    return m <= 96 ? cos384q(m) : -cos384q(192 - m);
}
__host__ __device__ constexpr double sin384(int m) { return cos384(96 - m); }

__host__ __device__ constexpr int imod(int a, int n) { return ((a % n) + n) % n; }

// b^-1 mod n for coprime b, n (small n: by search)
__host__ __device__ constexpr int inv_mod(int b, int n)
{
    for (int x = 1; x < n; x++)
        if (imod(b * x, n) == 1) return x;
    return n == 1 ? 0 : -1;
}

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev_n(int k, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((k >> b) & 1) << (bits - 1 - b);
    return r;
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E, typename F> __host__ __device__ __forceinline__ void sfor(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------- multiply by +-i

// forward direction: -i z; inverse: +i z
template <typename T, bool INV> __host__ __device__ __forceinline__ cx<T> mul_ni(cx<T> z)
{
    if constexpr (INV) return cx<T>{-z.im, z.re};
    else return cx<T>{z.im, -z.re};
}

// ---------------------------------------------------------------- butterflies

// x0 = a + w b, x1 = a - w b with w = w_N^E (exp(-2 pi i E/N) forward,
// conjugate inverse), N dividing 384.
template <typename T, int N, int E, bool INV>
__host__ __device__ __forceinline__ void bfly2(cx<T> a, cx<T> b, cx<T>& x0, cx<T>& x1)
{
    constexpr int e = imod(E, N);
    if constexpr (e == 0) {
        x0 = a + b;
        x1 = a - b;
    } else if constexpr (4 * e == N) {
        const cx<T> wb = mul_ni<T, INV>(b);  // w = -i forward
        x0 = a + wb;
        x1 = a - wb;
    } else if constexpr (2 * e == N) {
        x0 = a - b;
        x1 = a + b;
    } else if constexpr (4 * e == 3 * N) {
        const cx<T> wb = mul_ni<T, !INV>(b);  // w = +i forward
        x0 = a + wb;
        x1 = a - wb;
    } else {
        static_assert(384 % N == 0, "roots of unity of order dividing 384");
        constexpr int m = e * (384 / N);
        constexpr double wr = cos384(m);
        constexpr double wi = INV ? sin384(m) : -sin384(m);
        constexpr bool by_re = (wr < 0 ? -wr : wr) >= (wi < 0 ? -wi : wi);
        if constexpr (by_re) {
            // w b = wr (b_r - t b_i, b_i + t b_r), t = wi / wr
            constexpr T t = (T)(wi / wr), c = (T)wr;
            const T ur = fma(-t, b.im, b.re), ui = fma(t, b.re, b.im);
            x0 = cx<T>{fma(c, ur, a.re), fma(c, ui, a.im)};
            x1 = cx<T>{fma(-c, ur, a.re), fma(-c, ui, a.im)};
        } else {
            // w b = wi (t b_r - b_i, t b_i + b_r), t = wr / wi
            constexpr T t = (T)(wr / wi), c = (T)wi;
            const T ur = fma(t, b.re, -b.im), ui = fma(t, b.im, b.re);
            x0 = cx<T>{fma(c, ur, a.re), fma(c, ui, a.im)};
            x1 = cx<T>{fma(-c, ur, a.re), fma(-c, ui, a.im)};
        }
    }
}

// ---------------------------------------------------------------- codelets

template <typename T, int N, bool INV> __host__ __device__ __forceinline__ void dft(cx<T>* v);

template <typename T, bool INV> __host__ __device__ __forceinline__ void dft3(cx<T>* v)
{
    // X1 = c -+ i h (x1 - x2), X2 = c +- i h (x1 - x2), c = x0 - (x1 + x2)/2,
    // h = sqrt(3)/2 (upper signs forward)
    constexpr T h = (T)0.866025403784438646763723170752936183;
    const cx<T> t1 = v[1] + v[2], t2 = v[1] - v[2];
    const cx<T> c = cx<T>{fma((T)-0.5, t1.re, v[0].re), fma((T)-0.5, t1.im, v[0].im)};
    v[0] = v[0] + t1;
    constexpr T s = INV ? -h : h;  // X1 = c + s (t2_i, -t2_r)
    v[1] = cx<T>{fma(s, t2.im, c.re), fma(-s, t2.re, c.im)};
    v[2] = cx<T>{fma(-s, t2.im, c.re), fma(s, t2.re, c.im)};
}

template <typename T, bool INV> __host__ __device__ __forceinline__ void dft4(cx<T>* v)
{
    const cx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3];
    const cx<T> t3 = mul_ni<T, INV>(v[1] - v[3]);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
}

// prime-factor split N = A B, gcd(A, B) = 1: input index (B n1 + A n2) mod N,
// output index (B (B^-1 mod A) k1 + A (A^-1 mod B) k2) mod N
template <typename T, int A, int B, bool INV> __host__ __device__ __forceinline__ void dft_pfa(cx<T>* v)
{
    constexpr int N = A * B;
    cx<T> t[A][B];
    sfor<0, A>([&](auto n1) {
        sfor<0, B>([&](auto n2) { t[n1.value][n2.value] = v[imod(B * n1.value + A * n2.value, N)]; });
        dft<T, B, INV>(t[n1.value]);
    });
    constexpr int eb = B * inv_mod(B, A), ea = A * inv_mod(A, B);
    sfor<0, B>([&](auto k2) {
        cx<T> u[A];
        sfor<0, A>([&](auto n1) { u[n1.value] = t[n1.value][k2.value]; });
        dft<T, A, INV>(u);
        sfor<0, A>([&](auto k1) { v[imod(eb * k1.value + ea * k2.value, N)] = u[k1.value]; });
    });
}

// radix-2 decimation in time: X[k] = E[k] + w^k O[k], X[k + N/2] = E[k] - w^k O[k]
template <typename T, int N, bool INV> __host__ __device__ __forceinline__ void dft_r2(cx<T>* v)
{
    constexpr int M = N / 2;
    cx<T> e[M], o[M];
    sfor<0, M>([&](auto m) {
        e[m.value] = v[2 * m.value];
        o[m.value] = v[2 * m.value + 1];
    });
    dft<T, M, INV>(e);
    dft<T, M, INV>(o);
    sfor<0, M>([&](auto k) { bfly2<T, N, k.value, INV>(e[k.value], o[k.value], v[k.value], v[k.value + M]); });
}

template <typename T, int N, bool INV> __host__ __device__ __forceinline__ void dft(cx<T>* v)
{
    if constexpr (N == 1) {
    } else if constexpr (N == 2) {
        const cx<T> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    } else if constexpr (N == 3) {
        dft3<T, INV>(v);
    } else if constexpr (N == 4) {
        dft4<T, INV>(v);
    } else if constexpr (N % 3 == 0) {
        static_assert(is_pow2(N / 3), "codelet lengths are 2^k or 3 * 2^k");
        dft_pfa<T, N / 3, 3, INV>(v);
    } else {
        static_assert(is_pow2(N) && N <= 32, "codelet lengths are 2^k <= 32 or 3 * 2^k");
        dft_r2<T, N, INV>(v);
    }
}

// ---------------------------------------------------------------- lines

// lanes per line and values per lane of a line of length L.  FP64 (bound by the
// FP64 pipe: as few extra operations as possible): one lane up to 32 values;
// 48: two; 64, 96: four; 128: eight.  FP32 (bound by memory latency: more
// threads in flight, at the cost of cheap FP32 twiddles and shuffles): one lane
// up to 16; 24, 32, 48: two; 64, 96: four; 128: eight.
template <typename T> __host__ __device__ constexpr int line_lanes(int L)
{
    return sizeof(T) == 8 ? (L <= 32 ? 1 : L == 48 ? 2 : L == 128 ? 8 : 4)
                          : (L <= 16 ? 1 : L <= 48 ? 2 : L == 128 ? 8 : 4);
}
template <typename T> __host__ __device__ constexpr int line_vals(int L) { return L / line_lanes<T>(L); }

// lanes per line of a pass that holds one transform at a time (a forward or an
// inverse alone): FP32 lines up to 32 values fit one lane there
template <typename T> __host__ __device__ constexpr int pass_lanes(int L)
{
    return (sizeof(T) == 4 && L <= 32) ? 1 : line_lanes<T>(L);
}

__host__ __device__ constexpr bool line_length_ok(int L)
{
    return L == 4 || L == 6 || L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64 ||
           L == 96 || L == 128;
}

// Position (0..L-1) of the value a lane holds: before the forward transform
// (and after the inverse) element tau + T j; after the forward (and before the
// inverse) frequency r + R bitrev_T(tau).
template <typename T, int L, int NL = line_lanes<T>(L)> __host__ __device__ __forceinline__ int line_pos_x(int tau, int j)
{
    return tau + NL * j;
}
template <typename T, int L, int NL = line_lanes<T>(L)> __host__ __device__ __forceinline__ int line_pos_k(int tau, int r)
{
    return r + (L / NL) * bitrev_n(tau, ilog2(NL));
}

// w_L^(tau E) (forward; conjugate for the inverse) for the run-time lane index
// tau < T, chosen among T compile-time constants
template <typename T, int L, int Tl, int E, bool INV> __host__ __device__ __forceinline__ cx<T> lane_root(int tau)
{
    cx<T> w = cx<T>{(T)1, (T)0};
    sfor<1, Tl>([&](auto t) {
        constexpr int m = imod(t.value * E * (384 / L), 384);
        constexpr T c = (T)cos384(m), sn = (T)(INV ? sin384(m) : -sin384(m));
        if (tau == t.value) w = cx<T>{c, sn};
    });
    return w;
}

// steps 1-2 of the forward line transform in one lane (step 1 alone for T = 1)
template <typename T, int L, int NL = line_lanes<T>(L)>
__host__ __device__ __forceinline__ void line_fwd_local(cx<T>* v, int tau)
{
    constexpr int Tl = NL, R = L / Tl;
    dft<T, R, false>(v);
    if constexpr (Tl > 1) {
        sfor<1, R>([&](auto r) { v[r.value] = cmul(v[r.value], lane_root<T, L, Tl, r.value, false>(tau)); });
    }
}

// the inverse's last two steps: conjugate twiddles, then the R-point inverse codelet
template <typename T, int L, int NL = line_lanes<T>(L)>
__host__ __device__ __forceinline__ void line_inv_local(cx<T>* v, int tau)
{
    constexpr int Tl = NL, R = L / Tl;
    if constexpr (Tl > 1) {
        sfor<1, R>([&](auto r) { v[r.value] = cmul(v[r.value], lane_root<T, L, Tl, r.value, true>(tau)); });
    }
    dft<T, R, true>(v);
}

// sign flip of x when m is the sign mask (integer operations)
__host__ __device__ __forceinline__ double sflip(double x, unsigned m)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double(__double2hiint(x) ^ (int)m, __double2loint(x));
#else
    return m ? -x : x;
#endif
}
__host__ __device__ __forceinline__ float sflip(float x, unsigned m)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(__float_as_uint(x) ^ m);
#else
    return m ? -x : x;
#endif
}

// One radix-2 stage across lanes for lane bit h, o the partner lane's value
// (partner tau ^ h).  Forward (decimation in frequency): the low lane keeps
// v + o, the high lane o - v, then the high lane multiplies by w_2h^p,
// p = tau mod h (h = 1: 1; h = 2: 1 or -i, by exchanging and negating
// components; h = 4: w_8^p from the line's table).  Inverse (the stage undone,
// unnormalised): the high lane first multiplies by the conjugate root, then
// the same sums.
template <typename T>
__host__ __device__ __forceinline__ cx<T> xsum(cx<T> v, cx<T> o, int tau, int h)
{
    const unsigned m = (tau & h) ? 0x80000000u : 0u;
    return cx<T>{o.re + sflip(v.re, m), o.im + sflip(v.im, m)};
}

// multiply by -i (forward) or +i (inverse) in lanes where cond holds, by
// exchanging and negating components
template <typename T, int R, bool INV> __host__ __device__ __forceinline__ void xrot(cx<T>* v, bool cond)
{
#pragma unroll
    for (int r = 0; r < R; r++) {
        const T re = v[r].re, im = v[r].im;
        // forward -i z = (im, -re); inverse +i z = (-im, re)
        v[r].re = cond ? (INV ? sflip(im, 0x80000000u) : im) : re;
        v[r].im = cond ? (INV ? re : sflip(re, 0x80000000u)) : im;
    }
}

// the root step of stage h in every lane (forward: after the sums; inverse:
// conjugate, before the exchange): h = 2: -i in lanes with tau mod 4 = 3; h = 4:
// w_8^(tau mod 4) in lanes with bit 2 of tau set
template <typename T, int R, bool INV> __host__ __device__ __forceinline__ void xstage_root(cx<T>* v, int tau, int h)
{
    if (h == 2) {
        xrot<T, R, INV>(v, (tau & 3) == 3);
    } else if (h == 4) {
        const cx<T> w = lane_root<T, 8, 4, 1, INV>((tau & 4) ? (tau & 3) : 0);
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = cmul(v[r], w);
    }
}

#ifdef __CUDACC__
template <typename T> __device__ __forceinline__ cx<T> shfl_xor(cx<T> a, int d)
{
    return cx<T>{__shfl_xor_sync(0xffffffffu, a.re, d), __shfl_xor_sync(0xffffffffu, a.im, d)};
}

// Whole line transforms on the device.  Lanes of one line sit W = 32 / T lanes
// apart in the warp (lane = tau W + w); every lane of the warp must call.
template <typename T, int L, int NL = line_lanes<T>(L)> __device__ __forceinline__ void line_fwd(cx<T>* v, int tau)
{
    constexpr int Tl = NL, R = L / Tl, W = 32 / Tl;
    line_fwd_local<T, L, NL>(v, tau);
    if constexpr (Tl > 1) {
        sfor<0, ilog2(Tl)>([&](auto s) {
            constexpr int h = Tl >> (1 + s.value);
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = xsum(v[r], shfl_xor(v[r], h * W), tau, h);
            xstage_root<T, R, false>(v, tau, h);
        });
    }
}

template <typename T, int L, int NL = line_lanes<T>(L)> __device__ __forceinline__ void line_inv(cx<T>* v, int tau)
{
    constexpr int Tl = NL, R = L / Tl, W = 32 / Tl;
    if constexpr (Tl > 1) {
        sfor<0, ilog2(Tl)>([&](auto s) {
            constexpr int h = 1 << s.value;
            xstage_root<T, R, true>(v, tau, h);
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = xsum(v[r], shfl_xor(v[r], h * W), tau, h);
        });
    }
    line_inv_local<T, L, NL>(v, tau);
}
#endif

// Run f(std::integral_constant<int, L>) for the run-time line length L (one of
// the supported lengths up to LMAX); returns false for any other value.
template <int LMAX = 128, typename F> __host__ __device__ __forceinline__ bool with_length(int L, F&& f)
{
    if (L > LMAX) return false;
    if constexpr (LMAX <= 32) {
        switch (L) {
        case 4: f(std::integral_constant<int, 4>{}); return true;
        case 6: f(std::integral_constant<int, 6>{}); return true;
        case 8: f(std::integral_constant<int, 8>{}); return true;
        case 12: f(std::integral_constant<int, 12>{}); return true;
        case 16: f(std::integral_constant<int, 16>{}); return true;
        case 24: f(std::integral_constant<int, 24>{}); return true;
        case 32: f(std::integral_constant<int, 32>{}); return true;
        default: return false;
        }
    }
    switch (L) {
    case 4: f(std::integral_constant<int, 4>{}); return true;
    case 6: f(std::integral_constant<int, 6>{}); return true;
    case 8: f(std::integral_constant<int, 8>{}); return true;
    case 12: f(std::integral_constant<int, 12>{}); return true;
    case 16: f(std::integral_constant<int, 16>{}); return true;
    case 24: f(std::integral_constant<int, 24>{}); return true;
    case 32: f(std::integral_constant<int, 32>{}); return true;
    case 48: f(std::integral_constant<int, 48>{}); return true;
    case 64: f(std::integral_constant<int, 64>{}); return true;
    case 96: f(std::integral_constant<int, 96>{}); return true;
    case 128: f(std::integral_constant<int, 128>{}); return true;
    default: return false;
    }
}

}  // namespace lgf
