// One lattice over several ranks: the kernels and entry points of one rank's
// t-slab of the Fourier-accelerated iteration (FP64), the GPU counterpart of the
// paper's MPI code, whose 4D FFT is distributed by transposes.  The data
// exchanges between ranks (two halo planes and two all-to-all transposes per
// iteration) are the caller's: the entry points leave their inputs and outputs
// in device buffers of the slab (lgf_slab_buffer).
//
// Rank r of N holds the sites with t in [r nt, (r+1) nt), nt = Lt/N, in the
// library's site order (a slab is an Lx x Ly x Lz x nt lattice without wrap in t).
// Per iteration:
//   lgf_slab_pack_halo(AH): the packed anti-Hermitian parts of the t-links of the
//     slab's last plane -> send buffer (they enter the next slab's first plane);
//   lgf_slab_delta: Delta from the parts of the slab and of the previous slab's
//     last plane (halo receive buffer), theta and F of the slab, the x,y forward
//     transform, the z forward transform written in the all-to-all order of
//     buffer A (block j: the z-range [j nz, (j+1) nz) of every plane, nz = Lz/N);
//   (the caller moves A -> B by an all-to-all: block i of B is rank i's t-range
//     of this rank's z-range)
//   lgf_slab_accelerate: the t-lines of B forward, times p2max/(p2(k) V), back;
//   (the caller moves B -> A by the reverse all-to-all)
//   lgf_slab_build_g: the z inverse from A, the x,y inverse, g = reunit(1 +
//     alpha/2 Delta~); g of the slab's first plane -> halo send buffer (it is
//     g(x + t) of the previous slab's last plane);
//   lgf_slab_update: U <- g U g^dag(x + mu), g(x + t) of the last plane from the
//     halo receive buffer; G <- g G; the new links' packed parts for the next Delta.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lgf.h"
#include "lgf_kernels.cuh"
#include "lgf_launch.h"

namespace lgf {
namespace {

constexpr int kSlabThreads = 256;

// Delta of every slab site, one thread per site; the t-neighbour of the first
// plane comes from the halo plane ([4][Lz P], the previous slab's last plane).
__global__ void __launch_bounds__(kSlabThreads) k_slab_delta(Lat d, const double2* __restrict__ AH,
                                                             const double* __restrict__ Fs,
                                                             const double2* __restrict__ halo_ah,
                                                             double2* __restrict__ Fd, double* __restrict__ partials,
                                                             Ctl* ctl)
{
    const int V = d.V, PL = d.P * d.L[2];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double th = 0.0, fsum = 0.0;
    if (s < V) {
        int c[4];
        site_coords(d, s, c);
        cx<double> D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) D[k] = mk<double>(0.0, 0.0);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const bool from_halo = (mu == 3 && c[3] == 0);
            const int sb = from_halo ? s : site_shift(d, s, c[mu], mu, -1);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const cx<double> a = from_halo ? ld<double>(halo_ah + (size_t)k * PL + sb)
                                               : ld<double>(AH + (size_t)(mu * 4 + k) * V + sb);
                const cx<double> b = ld<double>(AH + (size_t)(mu * 4 + k) * V + s);
                D[k] = D[k] + (a - b);
            }
        }
        th = theta_site(D);
        fsum = Fs[s];
#pragma unroll
        for (int k = 0; k < 4; k++) st<double>(Fd + (size_t)k * V + s, D[k]);
    }
    reduce_theta_F(th, fsum, partials, ctl, nullptr, V);
}

// Lines along one axis held in global memory, nl of them, a contiguous chunk per
// block: the block's lines are [blockIdx.x * chunk, ...).
template <int LMAX, bool INV, typename LD, typename ST>
__device__ __forceinline__ void slab_lines(int len, int nl, int chunk, LD ld, ST st)
{
    const int l0 = (int)blockIdx.x * chunk;
    const int n = min(chunk, nl - l0);
    if (n <= 0) return;
    with_length<LMAX>(len, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        lines_pass<double, L, INV>(
            n, [&](int l, int e) { return ld(l0 + l, e); }, [&](int l, int e, cx<double> v) { st(l0 + l, e, v); });
    });
}

// z forward: lines (f, t, xy) of Fd [f][t][z][P] -> A [j][f][t][z - j nz][P]
__global__ void __launch_bounds__(128) k_slab_zfwd(Lat d, int nz, int chunk, const double2* __restrict__ Fd,
                                                   double2* __restrict__ A)
{
    const int P = d.P, Lz = d.L[2], nt = d.L[3], V = d.V;
    auto where = [&](int g, int& f, int& t, int& xy) {
        const int ft = (int)fdiv((unsigned)g, d.dP);
        xy = g - ft * P;
        f = ft / nt;
        t = ft - f * nt;
    };
    slab_lines<128, false>(
        Lz, 4 * nt * P, chunk,
        [&](int g, int e) {
            int f, t, xy;
            where(g, f, t, xy);
            return ldv<double>(Fd + (size_t)f * V + (size_t)(t * Lz + e) * P + xy);
        },
        [&](int g, int e, cx<double> v) {
            int f, t, xy;
            where(g, f, t, xy);
            const int j = e / nz, zj = e - j * nz;
            st<double>(A + ((((size_t)j * 4 + f) * nt + t) * nz + zj) * P + xy, v);
        });
}

// z inverse: lines (f, t, xy) of A [j][f][t][z - j nz][P] -> Fd [f][t][z][P]
__global__ void __launch_bounds__(128) k_slab_zinv(Lat d, int nz, int chunk, const double2* __restrict__ A,
                                                   double2* __restrict__ Fd)
{
    const int P = d.P, Lz = d.L[2], nt = d.L[3], V = d.V;
    auto where = [&](int g, int& f, int& t, int& xy) {
        const int ft = (int)fdiv((unsigned)g, d.dP);
        xy = g - ft * P;
        f = ft / nt;
        t = ft - f * nt;
    };
    slab_lines<128, true>(
        Lz, 4 * nt * P, chunk,
        [&](int g, int e) {
            int f, t, xy;
            where(g, f, t, xy);
            const int j = e / nz, zj = e - j * nz;
            return ldv<double>(A + ((((size_t)j * 4 + f) * nt + t) * nz + zj) * P + xy);
        },
        [&](int g, int e, cx<double> v) {
            int f, t, xy;
            where(g, f, t, xy);
            st<double>(Fd + (size_t)f * V + (size_t)(t * Lz + e) * P + xy, v);
        });
}

// t forward, multiplier, t inverse: lines (f, z, xy) of B [i][f][t - i nt][z][P],
// the multiplier table [kt][z][P] of this rank's z-range
__global__ void __launch_bounds__(128) k_slab_taccel(Lat d, int nz, int Lt, int chunk, double2* __restrict__ B,
                                                     const double* __restrict__ mult)
{
    const int P = d.P, nt = d.L[3];
    const int nl = 4 * nz * P;
    const int l0 = (int)blockIdx.x * chunk;
    const int n = min(chunk, nl - l0);
    if (n <= 0) return;
    auto where = [&](int g, int& f, int& z, int& xy) {
        const int fz = (int)fdiv((unsigned)g, d.dP);
        xy = g - fz * P;
        f = fz / nz;
        z = fz - f * nz;
    };
    auto at = [&](int g, int t) {
        int f, z, xy;
        where(g, f, z, xy);
        const int i = t / nt, ti = t - i * nt;
        return B + ((((size_t)i * 4 + f) * nt + ti) * nz + z) * P + xy;
    };
    with_length<128>(Lt, [&](auto Lc) {
        constexpr int L = decltype(Lc)::value;
        lines_accel<double, L>(
            n, [&](int l, int e) { return ldv<double>(at(l0 + l, e)); },
            [&](int l, int k) -> double {
                int f, z, xy;
                where(l0 + l, f, z, xy);
                return __ldg(mult + ((size_t)k * nz + z) * P + xy);
            },
            [&](int l, int e, cx<double> v) { st<double>(at(l0 + l, e), v); });
    });
}

// U <- g U g^dag(x + mu) and G <- g G, one thread per site; g(x + t) of the last
// plane from the halo plane ([9][Lz P], the next slab's first plane); the new
// links' packed parts (AH) and Re Tr per site (Fs) for the next Delta.
__global__ void __launch_bounds__(kSlabThreads) k_slab_update(Lat d, double2* __restrict__ U, double2* __restrict__ G,
                                                              const double2* __restrict__ g,
                                                              const double2* __restrict__ halo_g,
                                                              double2* __restrict__ AH, double* __restrict__ Fs)
{
    const int V = d.V, PL = d.P * d.L[2];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    site_coords(d, s, c);
    cx<double> gx[9];
    load_g<double>(g, V, s, gx);
    double f = 0.0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cx<double> u[9], gn[9], w[9], a[4];
        load_link<double>(U, V, d.ne, mu, s, u);
        if (mu == 3 && c[3] == d.L[3] - 1) {
            const int sp = s - (d.L[3] - 1) * PL;  // the site's place in a plane
#pragma unroll
            for (int e = 0; e < 9; e++) gn[e] = ld<double>(halo_g + (size_t)e * PL + sp);
        } else {
            load_g<double>(g, V, site_shift(d, s, c[mu], mu, +1), gn);
        }
        link_gug(gx, u, gn, w);
        store_link<double>(U, V, d.ne, mu, s, w);
        ah_pack(w, a);
#pragma unroll
        for (int k = 0; k < 4; k++) st<double>(AH + (size_t)(mu * 4 + k) * V + s, a[k]);
        f += w[0].re + w[4].re + w[8].re;
    }
    Fs[s] = f;
    gauge_accumulate<double>(G, V, s, gx);
}

// the multipliers p2max / (p2(k) V) of this rank's z-range, [kt][z - z0][P]
__global__ void k_slab_mult(int Lx, int P, int nz, int z0, int n, const double* __restrict__ s2x,
                            const double* __restrict__ s2y, const double* __restrict__ s2z,
                            const double* __restrict__ s2t, double p2max, double Vg, double* __restrict__ mult)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xy = i % P, r = i / P;
    const int z = r % nz, kt = r / nz;
    const int x = xy % Lx, y = xy / Lx;
    const double p2 = s2x[x] + s2y[y] + s2z[z0 + z] + s2t[kt];
    mult[i] = p2 > 0.0 ? p2max / (p2 * Vg) : 0.0;
}

}  // namespace
}  // namespace lgf

// ---------------------------------------------------------------- entry points

using namespace lgf;

#define SCK(call)                                   \
    do {                                            \
        if ((call) != cudaSuccess) return LGF_ERR_CUDA; \
    } while (0)

struct lgf_slab {
    int gdims[4];
    int nranks, rank, nt, nz;
    Lat d;         // the slab as an Lx x Ly x Lz x nt lattice (its t-wrap never used)
    Shape sh;
    Tables tb;
    cudaStream_t stream = nullptr;
    int nblk = 0;  // blocks of the per-site kernels
    bool have_links = false;
    double2 *U = nullptr, *G = nullptr, *g = nullptr, *AH = nullptr, *Fd = nullptr, *A = nullptr, *B = nullptr;
    double2 *ah_send = nullptr, *ah_recv = nullptr, *g_send = nullptr, *g_recv = nullptr;
    double *Fs = nullptr, *mult = nullptr, *s2 = nullptr, *partials = nullptr;
    unsigned long long* err = nullptr;
    Ctl* ctl = nullptr;
    // host images of the control block, one per writer: lgf_slab_delta's (read
    // back on return) and lgf_slab_build_g's, whose copy to the device may still be
    // queued when the caller returns; each is rewritten only after its previous
    // copy has run (lgf_slab_delta waits for the stream)
    Ctl* host_ctl = nullptr;
    Ctl* host_ctl_g = nullptr;
    cudaEvent_t ctl_g_copied = nullptr;  // recorded after the copy from host_ctl_g
};

namespace {

void slab_free(lgf_slab* c)
{
    void* ptrs[] = {c->U, c->G, c->g, c->AH, c->Fd, c->A, c->B, c->ah_send, c->ah_recv, c->g_send,
                    c->g_recv, c->Fs, c->mult, c->s2, c->partials, c->err, c->ctl};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->host_ctl) cudaFreeHost(c->host_ctl);
    if (c->host_ctl_g) cudaFreeHost(c->host_ctl_g);
    if (c->ctl_g_copied) cudaEventDestroy(c->ctl_g_copied);
}

bool supported_extent(int L)
{
    return L == 4 || L == 6 || L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64 || L == 96 ||
           L == 128;
}

// the control block of one stage, through the host image `img`: no stop
// condition (the caller decides), alpha
int slab_reset_ctl(lgf_slab* c, Ctl* img, double alpha)
{
    Ctl h;
    memset(&h, 0, sizeof h);
    h.alpha = alpha;
    h.tol = -1.0;
    h.tol_final = -1.0;
    h.max_iter = 0x7fffffff;
    h.phase = 1;
    *img = h;
    SCK(cudaMemcpyAsync(c->ctl, img, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    return LGF_OK;
}

}  // namespace

extern "C" int lgf_slab_create(const int gdims[4], int nranks, int rank, lgf_slab** out)
{
    if (!gdims || !out || nranks < 1 || rank < 0 || rank >= nranks) return LGF_ERR_ARG;
    *out = nullptr;
    for (int mu = 0; mu < 4; mu++)
        if (!supported_extent(gdims[mu])) return LGF_ERR_UNSUPPORTED_DIMS;
    if (gdims[3] % nranks || gdims[2] % nranks) return LGF_ERR_UNSUPPORTED_DIMS;
    const long long Vg = (long long)gdims[0] * gdims[1] * gdims[2] * gdims[3];
    if (24 * Vg >= (1LL << 31)) return LGF_ERR_UNSUPPORTED_DIMS;
    lgf_slab* c = new lgf_slab();
    memcpy(c->gdims, gdims, sizeof c->gdims);
    c->nranks = nranks;
    c->rank = rank;
    c->nt = gdims[3] / nranks;
    c->nz = gdims[2] / nranks;
    Lat& d = c->d;
    d.L[0] = gdims[0];
    d.L[1] = gdims[1];
    d.L[2] = gdims[2];
    d.L[3] = c->nt;
    d.stride[0] = 1;
    d.stride[1] = d.L[0];
    d.stride[2] = d.L[0] * d.L[1];
    d.stride[3] = d.L[0] * d.L[1] * d.L[2];
    d.P = d.L[0] * d.L[1];
    d.nplanes = d.L[2] * d.L[3];
    d.V = d.P * d.nplanes;
    d.ne = 6;
    lat_set_divisors(d);
    // the x,y plane tiles of FP64 (the slab's only tiled kernels)
    if (plane_tile_bytes(d, sizeof(double2)) > kTileBudget) {
        delete c;
        return LGF_ERR_UNSUPPORTED_DIMS;
    }
    c->sh.nt_xy = 128;
    c->sh.nt_zt = 128;
    c->sh.xw = 1;
    memset(&c->tb, 0, sizeof c->tb);
    const size_t V = (size_t)d.V, PL = (size_t)d.P * d.L[2];
    c->nblk = (int)((V + kSlabThreads - 1) / kSlabThreads);
    auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = al((void**)&c->U, 4 * 6 * V * sizeof(double2)) && al((void**)&c->G, 6 * V * sizeof(double2)) &&
              al((void**)&c->g, 9 * V * sizeof(double2)) && al((void**)&c->AH, 16 * V * sizeof(double2)) &&
              al((void**)&c->Fd, 4 * V * sizeof(double2)) && al((void**)&c->A, 4 * V * sizeof(double2)) &&
              al((void**)&c->B, 4 * V * sizeof(double2)) && al((void**)&c->ah_send, 4 * PL * sizeof(double2)) &&
              al((void**)&c->ah_recv, 4 * PL * sizeof(double2)) && al((void**)&c->g_send, 9 * PL * sizeof(double2)) &&
              al((void**)&c->g_recv, 9 * PL * sizeof(double2)) && al((void**)&c->Fs, V * sizeof(double)) &&
              al((void**)&c->mult, V * sizeof(double)) &&
              al((void**)&c->s2, (size_t)(gdims[0] + gdims[1] + gdims[2] + gdims[3]) * sizeof(double)) &&
              al((void**)&c->partials, 2 * (size_t)c->nblk * sizeof(double)) &&
              al((void**)&c->err, 3 * sizeof(unsigned long long)) && al((void**)&c->ctl, sizeof(Ctl)) &&
              cudaMallocHost((void**)&c->host_ctl, sizeof(Ctl)) == cudaSuccess &&
              cudaMallocHost((void**)&c->host_ctl_g, sizeof(Ctl)) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->ctl_g_copied, cudaEventDisableTiming) == cudaSuccess;
    if (!ok || prepare_kernels<double>(d, c->sh) != cudaSuccess) {
        slab_free(c);
        delete c;
        return LGF_ERR_CUDA;
    }
    // 4 sin^2(pi k / L) per axis of the whole lattice; p2max their maxima summed
    std::vector<double> s2;
    double p2max = 0.0;
    for (int mu = 0; mu < 4; mu++) {
        double m = 0.0;
        for (int k = 0; k < gdims[mu]; k++) {
            const double sn = std::sin(3.14159265358979323846 * k / gdims[mu]);
            const double v = 4.0 * sn * sn;
            s2.push_back(v);
            m = v > m ? v : m;
        }
        p2max += m;
    }
    const int n = (int)V;  // Lt * nz * P = V of the slab
    const double* s2x = c->s2;
    const double* s2y = s2x + gdims[0];
    const double* s2z = s2y + gdims[1];
    const double* s2t = s2z + gdims[2];
    if (cudaMemcpy(c->s2, s2.data(), s2.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        slab_free(c);
        delete c;
        return LGF_ERR_CUDA;
    }
    k_slab_mult<<<(n + 255) / 256, 256>>>(gdims[0], d.P, c->nz, rank * c->nz, n, s2x, s2y, s2z, s2t, p2max,
                                          (double)Vg, c->mult);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        slab_free(c);
        delete c;
        return LGF_ERR_CUDA;
    }
    *out = c;
    return LGF_OK;
}

extern "C" void lgf_slab_destroy(lgf_slab* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    slab_free(c);
    delete c;
}

extern "C" int lgf_slab_set_stream(lgf_slab* c, void* stream)
{
    if (!c) return LGF_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(stream);
    return LGF_OK;
}

extern "C" int lgf_slab_set_links(lgf_slab* c, const double* U)
{
    if (!c || !U) return LGF_ERR_ARG;
    const Lat& d = c->d;
    SCK(cudaMemsetAsync(c->err, 0, 3 * sizeof(unsigned long long), c->stream));
    launch_pack_links64(c->stream, d.V, d.ne, U, c->U, c->err);
    launch_identity_rows64(c->stream, d.V, c->G);
    SCK(cudaGetLastError());
    unsigned long long e[3];
    SCK(cudaMemcpyAsync(e, c->err, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    double eu, ed;
    memcpy(&eu, &e[0], sizeof eu);
    memcpy(&ed, &e[1], sizeof ed);
    if (!(eu < 1e-12) || !(ed < 1e-12)) return LGF_ERR_NOT_SU3;
    launch_ah_init<double>(d, c->stream, c->U, c->AH, c->Fs);
    SCK(cudaGetLastError());
    c->have_links = true;
    return LGF_OK;
}

extern "C" int lgf_slab_get_links(lgf_slab* c, double* U_out)
{
    if (!c || !U_out) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    launch_unpack_su3_64(c->stream, c->d.V, 4, c->d.ne, c->U, U_out);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(c->stream));
    return LGF_OK;
}

extern "C" int lgf_slab_get_gauge(lgf_slab* c, double* G_out)
{
    if (!c || !G_out) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    launch_unpack_su3_64(c->stream, c->d.V, 1, 6, c->G, G_out);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(c->stream));
    return LGF_OK;
}

extern "C" int lgf_slab_buffer(lgf_slab* c, int which, void** ptr, size_t* bytes)
{
    if (!c || !ptr || !bytes) return LGF_ERR_ARG;
    const size_t V = (size_t)c->d.V, PL = (size_t)c->d.P * c->d.L[2];
    switch (which) {
    case LGF_SLAB_A: *ptr = c->A; *bytes = 4 * V * sizeof(double2); break;
    case LGF_SLAB_B: *ptr = c->B; *bytes = 4 * V * sizeof(double2); break;
    case LGF_SLAB_AH_SEND: *ptr = c->ah_send; *bytes = 4 * PL * sizeof(double2); break;
    case LGF_SLAB_AH_RECV: *ptr = c->ah_recv; *bytes = 4 * PL * sizeof(double2); break;
    case LGF_SLAB_G_SEND: *ptr = c->g_send; *bytes = 9 * PL * sizeof(double2); break;
    case LGF_SLAB_G_RECV: *ptr = c->g_recv; *bytes = 9 * PL * sizeof(double2); break;
    default: return LGF_ERR_ARG;
    }
    return LGF_OK;
}

extern "C" int lgf_slab_pack_halo(lgf_slab* c, int which)
{
    if (!c) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    const size_t V = (size_t)c->d.V, PL = (size_t)c->d.P * c->d.L[2], row = PL * sizeof(double2);
    if (which == LGF_SLAB_AH_SEND) {
        // the four packed parts of the t-links (mu = 3) of the last plane
        const double2* src = c->AH + 12 * V + (size_t)(c->nt - 1) * PL;
        SCK(cudaMemcpy2DAsync(c->ah_send, row, src, V * sizeof(double2), row, 4, cudaMemcpyDeviceToDevice, c->stream));
    } else if (which == LGF_SLAB_G_SEND) {
        // the nine entries of g on the first plane
        SCK(cudaMemcpy2DAsync(c->g_send, row, c->g, V * sizeof(double2), row, 9, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        return LGF_ERR_ARG;
    }
    return LGF_OK;
}

extern "C" int lgf_slab_delta(lgf_slab* c, double* theta, double* F)
{
    if (!c) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    const Lat& d = c->d;
    int r = slab_reset_ctl(c, c->host_ctl, 0.0);
    if (r != LGF_OK) return r;
    k_slab_delta<<<c->nblk, kSlabThreads, 0, c->stream>>>(d, c->AH, c->Fs, c->ah_recv, c->Fd, c->partials, c->ctl);
    launch_xy_fft<double>(d, c->sh, c->tb, c->stream, c->Fd, false);
    const int chunk = 128, nl = 4 * d.L[3] * d.P;
    k_slab_zfwd<<<(nl + chunk - 1) / chunk, 128, 0, c->stream>>>(d, c->nz, chunk, c->Fd, c->A);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(c->host_ctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    if (theta) *theta = c->host_ctl->theta;
    if (F) *F = c->host_ctl->F;
    return LGF_OK;
}

extern "C" int lgf_slab_accelerate(lgf_slab* c)
{
    if (!c) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    const int chunk = 128, nl = 4 * c->nz * c->d.P;
    k_slab_taccel<<<(nl + chunk - 1) / chunk, 128, 0, c->stream>>>(c->d, c->nz, c->gdims[3], chunk, c->B, c->mult);
    SCK(cudaGetLastError());
    return LGF_OK;
}

extern "C" int lgf_slab_build_g(lgf_slab* c, double alpha)
{
    if (!c || !(alpha > 0)) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    const Lat& d = c->d;
    SCK(cudaEventSynchronize(c->ctl_g_copied));  // the previous call's copy has read the image
    int r = slab_reset_ctl(c, c->host_ctl_g, alpha);
    if (r != LGF_OK) return r;
    SCK(cudaEventRecord(c->ctl_g_copied, c->stream));
    const int chunk = 128, nl = 4 * d.L[3] * d.P;
    k_slab_zinv<<<(nl + chunk - 1) / chunk, 128, 0, c->stream>>>(d, c->nz, chunk, c->A, c->Fd);
    launch_xyinv_g<double>(d, c->sh, c->tb, c->stream, c->Fd, c->g, c->ctl);
    SCK(cudaGetLastError());
    return LGF_OK;
}

extern "C" int lgf_slab_update(lgf_slab* c)
{
    if (!c) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    k_slab_update<<<c->nblk, kSlabThreads, 0, c->stream>>>(c->d, c->U, c->G, c->g, c->g_recv, c->AH, c->Fs);
    SCK(cudaGetLastError());
    return LGF_OK;
}
