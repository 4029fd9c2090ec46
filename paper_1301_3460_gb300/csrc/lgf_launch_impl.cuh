// Definitions of the templated launchers of lgf_launch.h; included by the
// per-precision translation units, which instantiate them.
#pragma once
#include <cudaTypedefs.h>

#include <type_traits>

#include "lgf_aux.cuh"
#include "lgf_launch.h"
#include "lgf_tma.cuh"

namespace lgf {

// Line-length classes of the tiled kernels: every length (LMAX 128), and a
// variant for planes (both precisions) and FP32 pencils whose lines are all at
// most 32 long, which needs fewer registers (more warps per SM)
template <typename T> inline bool small_plane(const Lat& d) { return d.L[0] <= 32 && d.L[1] <= 32; }
template <typename T> inline bool small_pencil(const Lat& d) { return sizeof(T) == 4 && d.L[2] <= 32 && d.L[3] <= 32; }
// the TMA-staged z,t kernel has a variant for lines up to 32 in both precisions
inline bool short_zt_lines(const Lat& d) { return d.L[2] <= 32 && d.L[3] <= 32; }

// Tensor map of the four fields for the TMA-staged z,t kernel: dimensions
// (innermost first) x' (8-byte words, elem/8 per complex value), t, z, ky, field
// with the fields' byte strides, box {xw elem/8, Lt, Lz, 1, 1}.  The encoder is a
// host function of the driver (no device work); false if it is unavailable or
// refuses the layout.
inline bool make_pencil_tmap(const Lat& d, int xw, const void* Fd, size_t elem, CUtensorMap* tm)
{
    static PFN_cuTensorMapEncodeTiled_v12000 enc = []() {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (enc == nullptr) return false;
    const cuuint64_t cw = elem / 8, P = (cuuint64_t)d.P;
    const cuuint64_t gdim[5] = {(cuuint64_t)d.L[0] * cw, (cuuint64_t)d.L[3], (cuuint64_t)d.L[2], (cuuint64_t)d.L[1], 4};
    const cuuint64_t gstride[4] = {P * d.L[2] * elem, P * elem, (cuuint64_t)d.L[0] * elem, (cuuint64_t)d.V * elem};
    const cuuint32_t box[5] = {(cuuint32_t)(xw * cw), (cuuint32_t)d.L[3], (cuuint32_t)d.L[2], 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_INT64, 5, const_cast<void*>(Fd), gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


template <typename T> inline size_t xy_smem(const Lat& d) { return plane_smem_bytes(d, sizeof(vec2_t<T>)); }
template <typename T> inline size_t zt_smem(const Lat& d, const Shape& sh)
{
    return pencil_smem_bytes(d, sh.xw, sizeof(vec2_t<T>));
}

template <typename K> inline cudaError_t allow_max_smem(K* kernel, int optin)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// The dynamic shared-memory limit is a per-function attribute shared by every
// context in the process, so it is raised to the device's opt-in maximum (a
// permission, not a reservation) rather than to this lattice's need: a later
// context with smaller planes must not lower it under an earlier one.
template <typename T> cudaError_t prepare_kernels(const Lat& d, const Shape& sh)
{
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    if ((size_t)optin < xy_smem<T>(d) + 1024 || (size_t)optin < zt_smem<T>(d, sh)) return cudaErrorInvalidValue;
    if ((e = allow_max_smem(k_delta<T, true, 128>, optin))) return e;
    if ((e = allow_max_smem(k_delta<T, false, 128>, optin))) return e;
    if ((e = allow_max_smem(k_xyinv_g<T, T, 128>, optin))) return e;
    if ((e = allow_max_smem(k_xy_fft<T, false, 128>, optin))) return e;
    if ((e = allow_max_smem(k_xy_fft<T, true, 128>, optin))) return e;
    if ((e = allow_max_smem(k_zt<T, 128>, optin))) return e;
    if ((e = allow_max_smem(k_delta<T, true, 32>, optin))) return e;
    if ((e = allow_max_smem(k_xyinv_g<T, T, 32>, optin))) return e;
    if ((e = allow_max_smem(k_xy_fft<T, false, 32>, optin))) return e;
    if ((e = allow_max_smem(k_xy_fft<T, true, 32>, optin))) return e;
    if constexpr (sizeof(T) == 4) {
        if ((e = allow_max_smem(k_zt<T, 32>, optin))) return e;
    }
    if ((e = allow_max_smem(k_zt_tma<T, 32>, optin))) return e;
    if ((e = allow_max_smem(k_zt_tma<T, 128>, optin))) return e;
    return cudaSuccess;
}

// Grid of the TMA-staged z,t kernel for pencils of xw columns and nt threads: as
// many blocks as fit on the device at once, at most one per pencil; 0 when the
// form cannot run this shape (FP32 pencils narrower than two columns, shared
// memory beyond the tile budget, a tensor map the driver refuses).
template <typename T> int zt_tma_grid(const Lat& d, int nt, int xw)
{
    const size_t elem = sizeof(vec2_t<T>);
    if (xw * elem < 16) return 0;
    const size_t smem = zt_tma_smem_bytes(d, xw, elem);
    if (smem > kTileBudget) return 0;
    CUtensorMap tm;
    if (!make_pencil_tmap(d, xw, reinterpret_cast<const void*>((uintptr_t)4096), elem, &tm)) return 0;
    int dev = 0, optin = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))
        return 0;
    if (short_zt_lines(d)) {
        if (allow_max_smem(k_zt_tma<T, 32>, optin) ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_zt_tma<T, 32>, nt, smem))
            return 0;
    } else {
        if (allow_max_smem(k_zt_tma<T, 128>, optin) ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_zt_tma<T, 128>, nt, smem))
            return 0;
    }
    const int units = (d.L[0] / xw) * d.L[1] * 4;
    const long g = (long)per_sm * nsm;
    return (int)(g < units ? g : units);
}

template <typename T>
void launch_delta(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, const vec2_t<T>* AH, const T* Fs,
                  vec2_t<T>* Fd, double* partials, Ctl* ctl, double2* hist, bool fft)
{
    if (!fft)
        k_delta<T, false, 128><<<d.nplanes, sh.nt_xy, 0, s>>>(d, AH, Fs, Fd, partials, ctl, hist);
    else if (small_plane<T>(d))
        k_delta<T, true, 32><<<d.nplanes, sh.nt_xy, xy_smem<T>(d), s>>>(d, AH, Fs, Fd, partials, ctl, hist);
    else
        k_delta<T, true, 128><<<d.nplanes, sh.nt_xy, xy_smem<T>(d), s>>>(d, AH, Fs, Fd, partials, ctl, hist);
}

template <typename T> void launch_ah_init(const Lat& d, cudaStream_t s, const vec2_t<T>* U, vec2_t<T>* AH, T* Fs)
{
    k_ah_init<T><<<(d.V + 255) / 256, 256, 0, s>>>(d, U, AH, Fs);
}

template <typename T>
void launch_zt(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, vec2_t<T>* Fd, const Ctl* ctl)
{
    if (sh.zt_tma && sh.zt_grid > 0) {
        // the shape was checked against the same encoder (zt_tma_grid); a refusal
        // here (it cannot happen for the library's own buffers) leaves the
        // pencil-tiled kernel to do the same work
        CUtensorMap tm;
        if (make_pencil_tmap(d, sh.xw, Fd, sizeof(vec2_t<T>), &tm)) {
            const size_t smem = zt_tma_smem_bytes(d, sh.xw, sizeof(vec2_t<T>));
            Ctl* c = const_cast<Ctl*>(ctl);
            const float p2v = (float)(tb.p2max / d.V);
            if (short_zt_lines(d))
                k_zt_tma<T, 32><<<sh.zt_grid, sh.nt_zt, smem, s>>>(d, sh.xw, tm, c, tb.mult64, tb.s2f, p2v);
            else
                k_zt_tma<T, 128><<<sh.zt_grid, sh.nt_zt, smem, s>>>(d, sh.xw, tm, c, tb.mult64, tb.s2f, p2v);
            return;
        }
    }
    const dim3 grid(d.L[0] / sh.xw, d.L[1], 4);
    if constexpr (sizeof(T) == 4) {
        if (small_pencil<T>(d)) {
            k_zt<T, 32><<<grid, sh.nt_zt, zt_smem<T>(d, sh), s>>>(d, sh.xw, Fd, ctl, tb.mult64, tb.s2f,
                                                                  (float)(tb.p2max / d.V));
            return;
        }
    }
    k_zt<T, 128><<<grid, sh.nt_zt, zt_smem<T>(d, sh), s>>>(d, sh.xw, Fd, ctl, tb.mult64, tb.s2f,
                                                           (float)(tb.p2max / d.V));
}

template <typename T>
void launch_xyinv_g(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, const vec2_t<T>* Fd,
                    vec2_t<T>* g, const Ctl* ctl)
{
    if (small_plane<T>(d)) {
        k_xyinv_g<T, T, 32><<<d.nplanes, sh.nt_xy, xy_smem<T>(d), s>>>(d, Fd, g, ctl);
        return;
    }
    k_xyinv_g<T, T, 128><<<d.nplanes, sh.nt_xy, xy_smem<T>(d), s>>>(d, Fd, g, ctl);
}

template <typename T> void launch_build_g(const Lat& d, cudaStream_t s, const vec2_t<T>* Fd, vec2_t<T>* g, const Ctl* ctl)
{
    k_build_g<T, T><<<(d.V + 255) / 256, 256, 0, s>>>(d, Fd, g, ctl);
}

template <typename T>
void launch_xy_fft(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, vec2_t<T>* Fd, bool inv)
{
    const size_t sm = xy_smem<T>(d);
    if (small_plane<T>(d)) {
        if (inv)
            k_xy_fft<T, true, 32><<<d.nplanes, sh.nt_xy, sm, s>>>(d, Fd);
        else
            k_xy_fft<T, false, 32><<<d.nplanes, sh.nt_xy, sm, s>>>(d, Fd);
        return;
    }
    if (inv)
        k_xy_fft<T, true, 128><<<d.nplanes, sh.nt_xy, sm, s>>>(d, Fd);
    else
        k_xy_fft<T, false, 128><<<d.nplanes, sh.nt_xy, sm, s>>>(d, Fd);
}

template <typename T>
void launch_update(const Lat& d, cudaStream_t s, vec2_t<T>* U, vec2_t<T>* G, const vec2_t<T>* g, Ctl* ctl,
                   vec2_t<T>* AH, T* Fs)
{
    k_update<T><<<(d.V + 255) / 256, 256, 0, s>>>(d, U, G, g, ctl, AH, Fs);
}

#define LGF_INSTANTIATE(T)                                                                                        \
    template cudaError_t prepare_kernels<T>(const Lat&, const Shape&);                                           \
    template void launch_delta<T>(const Lat&, const Shape&, const Tables&, cudaStream_t, const vec2_t<T>*,       \
                                  const T*, vec2_t<T>*, double*, Ctl*, double2*, bool);                           \
    template void launch_ah_init<T>(const Lat&, cudaStream_t, const vec2_t<T>*, vec2_t<T>*, T*);                  \
    template void launch_zt<T>(const Lat&, const Shape&, const Tables&, cudaStream_t, vec2_t<T>*, const Ctl*);    \
    template int zt_tma_grid<T>(const Lat&, int, int);                                                            \
    template void launch_xyinv_g<T>(const Lat&, const Shape&, const Tables&, cudaStream_t, const vec2_t<T>*,     \
                                    vec2_t<T>*, const Ctl*);                                                      \
    template void launch_build_g<T>(const Lat&, cudaStream_t, const vec2_t<T>*, vec2_t<T>*, const Ctl*);          \
    template void launch_xy_fft<T>(const Lat&, const Shape&, const Tables&, cudaStream_t, vec2_t<T>*, bool);      \
    template void launch_update<T>(const Lat&, cudaStream_t, vec2_t<T>*, vec2_t<T>*, const vec2_t<T>*, Ctl*,       \
                                   vec2_t<T>*, T*);

}  // namespace lgf
