// FP32 instantiation of the iteration kernels (FP32 phase of the mixed mode), and
// the FP32 phase's fused update-and-Delta kernels.
#include "lgf_launch_impl.cuh"

namespace lgf {
LGF_INSTANTIATE(float)

int update_grid(int V) { return (V + 255) / 256; }

void launch_update_delta32(const Lat& d, cudaStream_t s, const float2* Uin, float2* Uout, float2* G, const float2* g,
                           Ctl* ctl, float2* Fd, double* partials, double2* hist)
{
    k_update_delta<float><<<update_grid(d.V), 256, 0, s>>>(d, Uin, Uout, G, g, ctl, Fd, partials, hist);
}

void launch_delta_links32(const Lat& d, cudaStream_t s, const float2* U, float2* Fd, double* partials, Ctl* ctl,
                          double2* hist, int every)
{
    k_delta_links<float><<<update_grid(d.V), 256, 0, s>>>(d, U, Fd, partials, ctl, hist, every);
}
}  // namespace lgf
