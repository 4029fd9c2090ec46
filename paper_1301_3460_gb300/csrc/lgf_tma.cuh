// z,t transform with TMA-staged pencils (forward FFT along z and t, the
// accelerator p2max/(p2(k) V) with the zero mode removed, inverse FFT along t and
// z; the paper's accelerated step, introduction).
//
// A persistent grid walks the pencils (x-chunk of xw columns, ky, field); each
// block holds two pencil buffers A0, A1 and one working tile B:
//   - one thread loads the next pencil into the idle buffer with one 5-D tensor
//     copy (cp.async.bulk.tensor), completing on that buffer's mbarrier, while the
//     block transforms the current one;
//   - the box is read in the order (x, t, z), so a buffer holds [z][t][xi] and the
//     z-lines of a warp (consecutive (t, xi)) sit in consecutive words;
//   - z forward: buffer -> registers -> B ([t][kz][xi], padded rows);
//     t forward, multiplier, t inverse: B in place;
//     z inverse: B -> registers -> the same buffer;
//   - the buffer goes back to the field with one tensor store (bulk group), and
//     is reloaded only after that store has finished reading it.
// Every wait on an mbarrier gives up after about a second of the GPU's global
// timer, sets Ctl::fault and stops the loop, so that a copy that never lands
// cannot hold the GPU.
#pragma once
#include <cuda.h>

#include "lgf_kernels.cuh"

namespace lgf {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of the given parity to complete; false after ~1 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 64; i++)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// 5-D tiled tensor copies: global -> shared (completing on an mbarrier) and
// shared -> global (bulk group)
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_5d(const CUtensorMap* tm, int c0, int c1, int c2, int c3, int c4,
                                             const void* src)
{
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
                     reinterpret_cast<unsigned long long>(tm)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every committed store has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store is complete
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// this thread's shared-memory writes become visible to the tensor copies
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared memory of the kernel: 128 bytes of alignment slack, two pencil buffers of
// xw Lz Lt values (each rounded up to 128 bytes), the working tile [t][kz][xi]
// (padded rows, see pencil_rs), FP32: the four tables of 4 sin^2(pi k/L), and two
// mbarriers.
__host__ __device__ inline size_t zt_tma_buf_bytes(const Lat& d, int xw, size_t elem)
{
    return ((size_t)xw * d.L[2] * d.L[3] * elem + 127) / 128 * 128;
}
__host__ __device__ inline size_t zt_tma_tile_bytes(const Lat& d, int xw, size_t elem)
{
    const size_t tile = (size_t)d.L[3] * pencil_rs(d, xw, elem) * elem;
    const size_t tables = elem == 8 ? (size_t)(d.L[0] + d.L[1] + d.L[2] + d.L[3]) * sizeof(float) : 0;
    return (tile + tables + 15) / 16 * 16;
}
__host__ __device__ inline size_t zt_tma_smem_bytes(const Lat& d, int xw, size_t elem)
{
    return 128 + 2 * zt_tma_buf_bytes(d, xw, elem) + zt_tma_tile_bytes(d, xw, elem) + 2 * sizeof(uint64_t);
}

// Units u = (xc, ky, f), xc fastest; pencils of xw columns (a power of two; FP32:
// at least 2, so that a box row is a multiple of 16 bytes).  The tensor map (see
// make_pencil_tmap) views the fields as [f][ky][z][t][x'] with x' counting 8-byte
// words (two per FP64 complex value) and has the box {xw words per value, Lt, Lz, 1, 1}.
template <typename T, int LMAX>
__global__ void __launch_bounds__(kTileMaxThreads<T>, kTileMinBlocks<T, LMAX>)
    k_zt_tma(Lat d, int xw, const __grid_constant__ CUtensorMap tmap, Ctl* ctl, const double* __restrict__ mult,
             const float* __restrict__ s2f, float p2max_v)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    if (ld_flag(&ctl->phase_done)) return;
    constexpr int cw = (int)(sizeof(vec2_t<T>) / 8);  // 8-byte words per complex value
    const int Lx = d.L[0], Ly = d.L[1], Lz = d.L[2], Lt = d.L[3];
    const int P = d.P;
    const int xs = __ffs(xw) - 1;
    const int nxc = Lx >> xs;
    const int nunits = nxc * Ly * 4;
    const int rs = pencil_rs(d, xw, sizeof(vec2_t<T>));
    const size_t abytes = zt_tma_buf_bytes(d, xw, sizeof(vec2_t<T>));
    const unsigned box_bytes = (unsigned)((size_t)xw * Lz * Lt * sizeof(vec2_t<T>));
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    auto buf = [&](int i) { return reinterpret_cast<vec2_t<T>*>(base + (i ? abytes : 0)); };
    vec2_t<T>* B = reinterpret_cast<vec2_t<T>*>(base + 2 * abytes);
    float* t32 = reinterpret_cast<float*>(B + (size_t)Lt * rs);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * abytes + zt_tma_tile_bytes(d, xw, sizeof(vec2_t<T>)));
    const CUtensorMap* tm = &tmap;

    float hc = 0.f;
    if constexpr (sizeof(T) == 4) {
        hc = 0.5f * (float)ctl->alpha * p2max_v;
        block_copy<4, float>(Lx + Ly + Lz + Lt, [&](int i) { return __ldg(s2f + i); },
                             [&](int i, float v) { t32[i] = v; });
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(tm)) : "memory");
    }
    __syncthreads();
    auto unit_coords = [&](int u, int& xc, int& ky, int& f) {
        xc = u % nxc;
        const int r = u / nxc;
        ky = r % Ly;
        f = r / Ly;
    };
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        int xc, ky, f;
        unit_coords(blockIdx.x, xc, ky, f);
        mbar_arrive_expect_tx(&bar[0], box_bytes);
        tma_load_5d(buf(0), tm, (xc << xs) * cw, 0, 0, ky, f, &bar[0]);
    }
    int k = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, k++) {
        const int sidx = k & 1;
        vec2_t<T>* A = buf(sidx);
        if (threadIdx.x == 0) {
            // the next pencil into the other buffer, once the store of its last
            // pencil has read it
            const int un = u + (int)gridDim.x;
            if (un < nunits) {
                int xc, ky, f;
                unit_coords(un, xc, ky, f);
                bulk_wait_read0();
                mbar_arrive_expect_tx(&bar[sidx ^ 1], box_bytes);
                tma_load_5d(buf(sidx ^ 1), tm, (xc << xs) * cw, 0, 0, ky, f, &bar[sidx ^ 1]);
            }
        }
        if (!mbar_wait_bounded(&bar[sidx], (unsigned)(k >> 1) & 1u)) s_abort = 1;
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) {
                atomicExch(&ctl->fault, 1);
                atomicExch(&ctl->phase_done, 1);
                atomicExch(&ctl->done, 1);
            }
            break;
        }
        int xc, ky, f;
        unit_coords(u, xc, ky, f);
        const int x0 = xc << xs;
        // z forward: lines (t, xi) from A ([z][t][xi]) to B ([t][kz][xi])
        with_length<LMAX>(Lz, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            lines_pass<T, L, false, line_lanes<T>(L)>(
                xw * Lt, [&](int l, int e) { return ldv<T>(A + (e * Lt * xw + l)); },
                [&](int l, int e, cx<T> v) {
                    const int tt = l >> xs, xi = l & (xw - 1);
                    st<T>(B + tt * rs + e * xw + xi, v);
                });
        });
        __syncthreads();
        // t forward, accelerator, t inverse: lines (kz, xi) of B, in place
        with_length<LMAX>(Lt, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            lines_accel<T, L>(
                xw * Lz, [&](int l, int e) { return ldv<T>(B + e * rs + l); },
                [&](int l, int kt) -> T {
                    const int kz = l >> xs, xi = l & (xw - 1);
                    if constexpr (sizeof(T) == 8) {
                        return __ldg(mult + (x0 + xi + Lx * ky + (size_t)P * (kz + Lz * kt)));
                    } else {
                        const float p2 = t32[x0 + xi] + t32[Lx + ky] + t32[Lx + Ly + kz] + t32[Lx + Ly + Lz + kt];
                        return p2 > 0.f ? __fdividef(hc, p2) : 0.f;
                    }
                },
                [&](int l, int e, cx<T> v) { st<T>(B + e * rs + l, v); });
        });
        __syncthreads();
        // z inverse: lines (t, xi) of B back to A in its [z][t][xi] order
        with_length<LMAX>(Lz, [&](auto Lc) {
            constexpr int L = decltype(Lc)::value;
            lines_pass<T, L, true, line_lanes<T>(L)>(
                xw * Lt,
                [&](int l, int e) {
                    const int tt = l >> xs, xi = l & (xw - 1);
                    return ldv<T>(B + tt * rs + e * xw + xi);
                },
                [&](int l, int e, cx<T> v) { st<T>(A + (e * Lt * xw + l), v); });
        });
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_5d(tm, x0 * cw, 0, 0, ky, f, A);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) bulk_wait0();
}

}  // namespace lgf
