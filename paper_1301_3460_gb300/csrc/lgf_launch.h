// Host-side launch interface between the C ABI (lgf_capi.cu) and the kernel
// translation units (lgf_k64.cu: FP64 kernels and the conversion kernels,
// lgf_k32.cu: FP32 kernels, lgf_wilson.cu: configuration generation).  Splitting by precision keeps each unit small and
// lets them compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "lgf_common.cuh"

namespace lgf {

// per-axis twiddle tables exp(-2 pi i m / L_mu), momentum table 4 sin^2(pi k / L_mu)
struct Tables {
    const double2* tw64[4];
    const float2* tw32[4];
    const double* s2[4];
    double p2max;
    const double* mult64;  // p2max/(p2(k) V) per momentum (site-indexed)
    const float* mult32;
    const float* s2f;      // the four tables 4 sin^2(pi k / L_mu) in FP32, one after the other
};

// launch shape of the tiled FFT kernels of one precision
struct Shape {
    int nt_xy = 0;    // threads of the xy-plane kernels (a multiple of 32, at most 256)
    int nt_zt = 0;    // threads of the zt-pencil kernel (likewise)
    int xw = 0;       // x-columns per zt pencil (divides Lx)
    int zt_tma = 0;   // z,t kernel: 0 one block per pencil, 1 persistent with TMA-staged pencils
    int zt_grid = 0;  // blocks of the persistent form (zt_tma_grid)
};

// shared memory of the plane tile and of one pencil (element size elem)
size_t plane_tile_bytes(const Lat& d, size_t elem);
size_t pencil_tile_bytes(const Lat& d, int xw, size_t elem);
// shared-memory budget of one tile; extents whose tiles exceed it are refused
constexpr size_t kTileBudget = 220 * 1024;

template <typename T> cudaError_t prepare_kernels(const Lat& d, const Shape& sh);
template <typename T>
void launch_delta(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, const vec2_t<T>* AH, const T* Fs,
                  vec2_t<T>* Fd, double* partials, Ctl* ctl, double2* hist, bool fft);
template <typename T> void launch_ah_init(const Lat& d, cudaStream_t s, const vec2_t<T>* U, vec2_t<T>* AH, T* Fs);
template <typename T>
void launch_zt(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, vec2_t<T>* Fd, const Ctl* ctl);
// blocks of the TMA-staged z,t kernel for this lattice, nt threads and pencils
// of xw columns (0: the form cannot run that shape)
template <typename T> int zt_tma_grid(const Lat& d, int nt, int xw);
template <typename T>
void launch_xyinv_g(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, const vec2_t<T>* Fd,
                    vec2_t<T>* g, const Ctl* ctl);
template <typename T> void launch_build_g(const Lat& d, cudaStream_t s, const vec2_t<T>* Fd, vec2_t<T>* g, const Ctl* ctl);
template <typename T>
void launch_xy_fft(const Lat& d, const Shape& sh, const Tables& tb, cudaStream_t s, vec2_t<T>* Fd, bool inv);
template <typename T>
void launch_update(const Lat& d, cudaStream_t s, vec2_t<T>* U, vec2_t<T>* G, const vec2_t<T>* g, Ctl* ctl,
                   vec2_t<T>* AH, T* Fs);
// FP32 phase: the update fused with Delta, theta and F (links Uin -> Uout, Delta
// in space to Fd), and Delta, theta and F of stored links (every > 0: only on
// the FP32 phase's refresh iterations); grids of update_grid(V) blocks
int update_grid(int V);
void launch_update_delta32(const Lat& d, cudaStream_t s, const float2* Uin, float2* Uout, float2* G, const float2* g,
                           Ctl* ctl, float2* Fd, double* partials, double2* hist);
void launch_delta_links32(const Lat& d, cudaStream_t s, const float2* U, float2* Fd, double* partials, Ctl* ctl,
                          double2* hist, int every);

// FP32 phase: the g builder and the update in one persistent launch (k_gu); sync
// holds 4 + Lz Lt words, zeroed once before the first launch.  gu32_prepare
// raises the kernel's shared-memory limit.
cudaError_t gu32_prepare(const Lat& d);
void launch_gu32(const Lat& d, const Shape& sh, cudaStream_t s, const float2* Fd, float2* g, float2* U, float2* G,
                 float2* AH, float* Fs, Ctl* ctl, unsigned* sync);

// FP64 iterations with the accelerator in FP32 (FP64 unit): Delta, theta and F
// from the FP64 packed parts with the forward x,y transform in FP32 (Fd32), and
// the FP32 inverse x,y transform with the FP64 Gram-Schmidt writing an FP64 g;
// the FP32 z,t kernel (launch_zt<float>) sits between them
cudaError_t prepare_accel32(const Lat& d);
void launch_delta64_f32(const Lat& d, const Shape& sh64, cudaStream_t s, const double2* AH, const double* Fs,
                        float2* Fd, double* partials, Ctl* ctl, double2* hist);
void launch_xyinv_g32_64(const Lat& d, const Shape& sh32, cudaStream_t s, const float2* Fd, double2* g,
                         const Ctl* ctl);

// conversion, checking and mode-switch kernels (FP64 unit)
void launch_pack_links64(cudaStream_t s, int V, int ne, const double* in, double2* U, unsigned long long* err);
void launch_unpack_su3_64(cudaStream_t s, int V, int nmat, int ne, const double2* U, double* out);
void launch_identity_rows64(cudaStream_t s, int V, double2* G);
void launch_pack_delta(cudaStream_t s, int V, const double* in, double2* Fd);
void launch_unpack_delta(cudaStream_t s, int V, const double2* Fd, double* out);
void launch_unpack_full(cudaStream_t s, int V, const double2* g, double* out);
// n complex values FP64 -> FP32 and FP32 -> FP64, times scale
void launch_planes_to32(cudaStream_t s, long n, const double2* in, float2* out, double scale);
void launch_planes_to64(cudaStream_t s, long n, const float2* in, double2* out, double scale);
void launch_mixed_prep(cudaStream_t s, int V, int ne, const double2* U64, float2* U32, float2* G32, const Ctl* ctl);
void launch_switch(cudaStream_t s, const Lat& d, const float2* G32, double2* Gs, double2* U64, double2* G64,
                   Ctl* ctl);
void launch_loop_ctl(cudaStream_t s, Ctl* ctl, cudaGraphConditionalHandle h);
// FP32 phase: every `every` updates, G re-orthonormalised and U32 rebuilt as G U_in G^dag
void launch_refresh32(cudaStream_t s, const Lat& d32, int ne64, const double2* U64, float2* G32, float2* U32,
                      float2* AH32, float* Fs32, const Ctl* ctl, int every);
void launch_make_mult(cudaStream_t s, const Lat& d, const Tables& tb, double* m64, float* m32);
// derivative of one step and of the gluon propagator (lgf_diff.cuh)
void launch_g_from_dt(cudaStream_t s, int V, const double2* Fd, double2* g, double alpha);
void launch_pack_full(cudaStream_t s, int V, const double* in, double2* out);
void launch_unpack_planes(cudaStream_t s, int V, const double2* in, double* out);
void launch_step_bwd(cudaStream_t s, const Lat& d, const double2* U, const double2* g, const double2* Fdt,
                     double2* Gp, double2* Gud, double2* Ggs, double2* Q, double alpha, double2* FA, double2* FB);
void launch_bwd_delta(cudaStream_t s, const Lat& d, const double2* U, const double2* FA, const double2* FB,
                      const double2* Gud, double2* Gin);
int gluon_blocks(int V);
void launch_gluon(cudaStream_t s, const Lat& d, const double2* U, const Tables& tb, double2* part, double2* At,
                  double* D);
void launch_gluon_bwd(cudaStream_t s, const Lat& d, const double2* U, const double2* At, double coef, const Tables& tb,
                      double2* Gout);
// Wilson-action heat bath / overrelaxation of one (mu, parity) class of links,
// and the mean plaquette (lgf_wilson.cu)
void launch_wilson(cudaStream_t s, const Lat& d, double2* U, float2* U32, int mu, int parity, int overrelax,
                   double beta, unsigned long long seed, unsigned int sweep, int precision);
void launch_links_to_fp32(cudaStream_t s, const Lat& d, const double2* U, float2* U32);
void launch_unit_links(cudaStream_t s, const Lat& d, double2* U);
int plaquette_blocks(int V);
void launch_plaquette(cudaStream_t s, const Lat& d, const double2* U, double* part, double* out);
// writes the GPU's global nanosecond timer to *p
void launch_stamp(cudaStream_t s, unsigned long long* p);

}  // namespace lgf
