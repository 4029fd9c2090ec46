// FP64 instantiation of the iteration kernels, plus the conversion, input-check
// and precision-switch kernels (all FP64).
#include "lgf_diff.cuh"
#include "lgf_launch_impl.cuh"

namespace lgf {

LGF_INSTANTIATE(double)

size_t plane_tile_bytes(const Lat& d, size_t elem) { return plane_smem_bytes(d, elem); }
size_t pencil_tile_bytes(const Lat& d, int xw, size_t elem) { return pencil_smem_bytes(d, xw, elem); }

namespace {
inline unsigned blocks(long n, int nt) { return (unsigned)((n + nt - 1) / nt); }
}  // namespace

cudaError_t prepare_accel32(const Lat& d)
{
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    if ((size_t)optin < plane_smem_bytes(d, sizeof(float2)) + 1024) return cudaErrorInvalidValue;
    if ((e = allow_max_smem(k_delta<double, true, 32, float>, optin))) return e;
    if ((e = allow_max_smem(k_delta<double, true, 128, float>, optin))) return e;
    if ((e = allow_max_smem(k_xyinv_g<float, double, 32>, optin))) return e;
    if ((e = allow_max_smem(k_xyinv_g<float, double, 128>, optin))) return e;
    return cudaSuccess;
}

void launch_delta64_f32(const Lat& d, const Shape& sh64, cudaStream_t s, const double2* AH, const double* Fs,
                        float2* Fd, double* partials, Ctl* ctl, double2* hist)
{
    const size_t sm = plane_smem_bytes(d, sizeof(float2));
    if (small_plane<double>(d))
        k_delta<double, true, 32, float><<<d.nplanes, sh64.nt_xy, sm, s>>>(d, AH, Fs, Fd, partials, ctl, hist);
    else
        k_delta<double, true, 128, float><<<d.nplanes, sh64.nt_xy, sm, s>>>(d, AH, Fs, Fd, partials, ctl, hist);
}

void launch_xyinv_g32_64(const Lat& d, const Shape& sh32, cudaStream_t s, const float2* Fd, double2* g,
                         const Ctl* ctl)
{
    const size_t sm = plane_smem_bytes(d, sizeof(float2));
    if (small_plane<float>(d))
        k_xyinv_g<float, double, 32><<<d.nplanes, sh32.nt_xy, sm, s>>>(d, Fd, g, ctl);
    else
        k_xyinv_g<float, double, 128><<<d.nplanes, sh32.nt_xy, sm, s>>>(d, Fd, g, ctl);
}

void launch_pack_links64(cudaStream_t s, int V, int ne, const double* in, double2* U, unsigned long long* err)
{
    k_pack_links<double><<<blocks(4L * V, 256), 256, 0, s>>>(V, ne, in, U, err, 1);
}
void launch_unpack_su3_64(cudaStream_t s, int V, int nmat, int ne, const double2* U, double* out)
{
    k_unpack_su3<double><<<blocks((long)nmat * V, 256), 256, 0, s>>>(V, nmat, ne, U, out);
}
void launch_identity_rows64(cudaStream_t s, int V, double2* G)
{
    k_identity_rows<double><<<blocks(V, 256), 256, 0, s>>>(V, G);
}
void launch_pack_delta(cudaStream_t s, int V, const double* in, double2* Fd)
{
    k_pack_delta<<<blocks(V, 256), 256, 0, s>>>(V, in, Fd);
}
void launch_unpack_delta(cudaStream_t s, int V, const double2* Fd, double* out)
{
    k_unpack_delta<<<blocks(V, 256), 256, 0, s>>>(V, Fd, out);
}
void launch_unpack_full(cudaStream_t s, int V, const double2* g, double* out)
{
    k_unpack_full<<<blocks(V, 256), 256, 0, s>>>(V, g, out);
}
void launch_planes_to32(cudaStream_t s, long n, const double2* in, float2* out, double scale)
{
    k_planes_to32<<<blocks(n, 256), 256, 0, s>>>(n, in, out, scale);
}
void launch_planes_to64(cudaStream_t s, long n, const float2* in, double2* out, double scale)
{
    k_planes_to64<<<blocks(n, 256), 256, 0, s>>>(n, in, out, scale);
}
void launch_mixed_prep(cudaStream_t s, int V, int ne, const double2* U64, float2* U32, float2* G32, const Ctl* ctl)
{
    k_mixed_prep<<<blocks(V, 256), 256, 0, s>>>(V, ne, U64, U32, G32, ctl);
}
void launch_switch(cudaStream_t s, const Lat& d, const float2* G32, double2* Gs, double2* U64, double2* G64,
                   Ctl* ctl)
{
    k_switch_gs<<<blocks(d.V, 256), 256, 0, s>>>(d.V, G32, Gs, ctl);
    k_project<<<blocks(d.V, 256), 256, 0, s>>>(d, U64, G64, Gs, ctl);
    k_phase_switch<<<1, 1, 0, s>>>(ctl);
}
void launch_refresh32(cudaStream_t s, const Lat& d32, int ne64, const double2* U64, float2* G32, float2* U32,
                      float2* AH32, float* Fs32, const Ctl* ctl, int every)
{
    k_refresh_g<<<blocks(d32.V, 256), 256, 0, s>>>(d32.V, G32, ctl, every);
    k_refresh_u<<<blocks(d32.V, 256), 256, 0, s>>>(d32, ne64, U64, G32, U32, AH32, Fs32, ctl, every);
}
static __global__ void k_stamp(unsigned long long* p)
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    *p = t;
}
void launch_stamp(cudaStream_t s, unsigned long long* p) { k_stamp<<<1, 1, 0, s>>>(p); }

void launch_make_mult(cudaStream_t s, const Lat& d, const Tables& tb, double* m64, float* m32)
{
    k_make_mult<<<blocks(d.V, 256), 256, 0, s>>>(d, tb.s2[0], tb.s2[1], tb.s2[2], tb.s2[3], tb.p2max, m64, m32);
}
void launch_g_from_dt(cudaStream_t s, int V, const double2* Fd, double2* g, double alpha)
{
    k_g_from_dt<<<blocks(V, 256), 256, 0, s>>>(V, Fd, g, alpha);
}
void launch_pack_full(cudaStream_t s, int V, const double* in, double2* out)
{
    k_pack_full<<<blocks(4L * V, 256), 256, 0, s>>>(V, in, out);
}
void launch_unpack_planes(cudaStream_t s, int V, const double2* in, double* out)
{
    k_unpack_planes<<<blocks(4L * V, 256), 256, 0, s>>>(V, in, out);
}
void launch_step_bwd(cudaStream_t s, const Lat& d, const double2* U, const double2* g, const double2* Fdt,
                     double2* Gp, double2* Gud, double2* Ggs, double2* Q, double alpha, double2* FA, double2* FB)
{
    k_bwd_update<<<blocks(d.V, 128), 128, 0, s>>>(d, U, g, Gp, Gud, Ggs, Q);
    k_bwd_reunit<<<blocks(d.V, 256), 256, 0, s>>>(d, Fdt, Ggs, Q, alpha, FA, FB);
}
void launch_bwd_delta(cudaStream_t s, const Lat& d, const double2* U, const double2* FA, const double2* FB,
                      const double2* Gud, double2* Gin)
{
    k_bwd_delta<<<blocks(d.V, 256), 256, 0, s>>>(d, U, FA, FB, Gud, Gin);
}
int gluon_blocks(int V) { int nb = (V + 255) / 256; return nb < 608 ? nb : 608; }
void launch_gluon(cudaStream_t s, const Lat& d, const double2* U, const Tables& tb, double2* part, double2* At,
                  double* D)
{
    const int nbx = gluon_blocks(d.V);
    k_gluon_partial<<<dim3(nbx, 16), 256, 0, s>>>(d, U, tb.tw64[0], tb.tw64[1], tb.tw64[2], tb.tw64[3], part);
    const double c = 2.0 / (8.0 * 3.0 * (double)d.V);
    k_gluon_final<<<1, 160, 0, s>>>(nbx, c, part, At, D);
}
void launch_gluon_bwd(cudaStream_t s, const Lat& d, const double2* U, const double2* At, double coef, const Tables& tb,
                      double2* Gout)
{
    k_gluon_bwd<<<blocks(d.V, 256), 256, 0, s>>>(d, U, At, coef, tb.tw64[0], tb.tw64[1], tb.tw64[2], tb.tw64[3], Gout);
}

void launch_loop_ctl(cudaStream_t s, Ctl* ctl, cudaGraphConditionalHandle h)
{
    k_loop_ctl<<<1, 1, 0, s>>>(ctl, h, 0x7fffffffu);
}

}  // namespace lgf
