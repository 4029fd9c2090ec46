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

cudaError_t gu32_prepare(const Lat& d)
{
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    if ((e = allow_max_smem(k_gu<float, 32>, optin))) return e;
    return allow_max_smem(k_gu<float, 128>, optin);
}

// Blocks of 256 threads whatever the plane kernels' shape (measured on GB300:
// 242 against 280 us for the 32^4 g builder and update at 128 threads, where the
// two-kernel form takes 252-254 us at either size); grid: the blocks the device
// holds at once (a persistent launch); lag of the queue: the resident blocks
// over Lz t-steps (twice as many items as blocks; measured on GB300 against
// fixed lags 1-48: within 1% of the best at 32^4, 48^4 and 32^3x64, and 3-4%
// faster than half of it).
void launch_gu32(const Lat& d, const Shape&, cudaStream_t s, const float2* Fd, float2* g, float2* U, float2* G,
                 float2* AH, float* Fs, Ctl* ctl, unsigned* sync)
{
    constexpr int nt = 256;
    const size_t sm = xy_smem<float>(d);
    const bool small = small_plane<float>(d);
    int dev = 0, nsm = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (small)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gu<float, 32>, nt, sm);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gu<float, 128>, nt, sm);
    if (per_sm < 1) per_sm = 1;
    int grid = per_sm * nsm;
    if (grid > 2 * d.nplanes) grid = 2 * d.nplanes;
    const int Lz = d.L[2], Lt = d.L[3];
    int lag = (grid + Lz - 1) / Lz;
    lag = lag < 1 ? 1 : (lag > Lt ? Lt : lag);
    if (small)
        k_gu<float, 32><<<grid, nt, sm, s>>>(d, Fd, g, U, G, AH, Fs, ctl, sync, lag);
    else
        k_gu<float, 128><<<grid, nt, sm, s>>>(d, Fd, g, U, G, AH, Fs, ctl, sync, lag);
}

void launch_delta_links32(const Lat& d, cudaStream_t s, const float2* U, float2* Fd, double* partials, Ctl* ctl,
                          double2* hist, int every)
{
    k_delta_links<float><<<update_grid(d.V), 256, 0, s>>>(d, U, Fd, partials, ctl, hist, every);
}
}  // namespace lgf
