// lgf_accelerate_noalloc: the Fourier-acceleration stage for callers that
// cannot allocate device memory.
//
// Some callers hand all of the GPU's memory to an allocator of their own (a
// framework's caching pool, an embedded runtime with one fixed arena) and have
// nothing left to give a library that calls cudaMalloc; lgf_create allocates a
// context, so they cannot use lgf_accelerate.  This entry point runs the same
// kernels with its scratch (the four packed colour fields, the twiddle and
// momentum tables, the accelerator's multiplier table and the small control
// block) in a file-scope device array, so the call itself allocates nothing:
// the caller passes only the input and output buffers.
//
// The array is sized for lattices of up to kMaxSites sites (4 MiB of fields,
// 0.75 MiB of multipliers and the small tables), is part of the loaded module
// and is therefore held on every GPU that loads the library until the process
// exits.  All calls share it and it keeps
// the last call's contents; the control block is cleared on every call and the
// fields and tables are overwritten before use.  Two calls whose work overlaps
// on the GPU (different streams, or different host threads on one device) race
// on the array.
//
// The array's device address is looked up on every call (a lookup allocates
// nothing): after cudaDeviceReset, or from another context on the same device,
// the module is loaded again and the array can move, so a cached address could
// point into memory the caller owns.  The kernel attributes are set on the
// first call on a device and again whenever the address has changed.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/lgf.h"
#include "lgf_dft.cuh"
#include "lgf_launch.h"

using namespace lgf;

namespace {

constexpr int kMaxSites = 65536;  // e.g. 16^4
constexpr int kMaxLen = 128;
constexpr size_t kFieldBytes = (size_t)4 * kMaxSites * sizeof(double2);
constexpr size_t kTw64Bytes = (size_t)4 * kMaxLen * sizeof(double2);
constexpr size_t kTw32Bytes = (size_t)4 * kMaxLen * sizeof(float2);
constexpr size_t kS2Bytes = (size_t)4 * kMaxLen * sizeof(double);
constexpr size_t kMultBytes = (size_t)kMaxSites * (sizeof(double) + sizeof(float));  // accelerator table, FP64 + FP32
constexpr size_t kTablesOff = kFieldBytes;
constexpr size_t kMultOff = (kTablesOff + kTw64Bytes + kTw32Bytes + kS2Bytes + 255) / 256 * 256;
constexpr size_t kCtlOff = (kMultOff + kMultBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCtlOff + (sizeof(Ctl) + 255) / 256 * 256;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
unsigned char* g_scratch[kMaxDevices] = {};  // device address at the last set-up, per device

bool length_ok(int L) { return line_length_ok(L); }

}  // namespace

static __device__ __align__(256) unsigned char lgf_noalloc_scratch[kScratchBytes];

extern "C" int lgf_accelerate_noalloc(const int dims[4], const double* Delta_in, double* Dt_out, void* cuda_stream)
{
    if (!dims || !Delta_in || !Dt_out) return LGF_ERR_ARG;
    long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (!length_ok(dims[mu])) return LGF_ERR_UNSUPPORTED_DIMS;
        V *= dims[mu];
    }
    if (V > kMaxSites) return LGF_ERR_UNSUPPORTED_DIMS;  // larger lattices need lgf_create + lgf_accelerate

    Lat d{};
    int st = 1;
    for (int mu = 0; mu < 4; mu++) {
        d.L[mu] = dims[mu];
        d.stride[mu] = st;
        st *= dims[mu];
    }
    d.V = (int)V;
    d.P = dims[0] * dims[1];
    d.nplanes = dims[2] * dims[3];
    lat_set_divisors(d);
    // FFT tiles in shared memory: the four fields of an xy-plane, and one z,t
    // pencil of up to four x-columns
    if (plane_tile_bytes(d, sizeof(double2)) > kTileBudget) return LGF_ERR_UNSUPPORTED_DIMS;
    Shape sh{};
    sh.nt_xy = 128;
    sh.nt_zt = 128;
    sh.xw = 4;
    while (sh.xw > 1 && (dims[0] % sh.xw || pencil_tile_bytes(d, sh.xw, sizeof(double2)) > kTileBudget)) sh.xw >>= 1;
    if (pencil_tile_bytes(d, sh.xw, sizeof(double2)) > kTileBudget) return LGF_ERR_UNSUPPORTED_DIMS;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LGF_ERR_CUDA;
    unsigned char* base;
    {
        // With the device current: the host-side name of the array is not a device
        // address, so take the address from the runtime, on every call.  Set-up
        // (kernel attributes) on the first call on this device and whenever the
        // address differs from the one seen at the last set-up.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, lgf_noalloc_scratch) != cudaSuccess || !p) return LGF_ERR_CUDA;
        if (g_scratch[dev] != static_cast<unsigned char*>(p)) {
            if (prepare_kernels<double>(d, sh) != cudaSuccess) return LGF_ERR_CUDA;
            g_scratch[dev] = static_cast<unsigned char*>(p);
        }
        base = static_cast<unsigned char*>(p);
    }

    // tables for these extents, written into the array (host copies on the stack)
    double2 tw64[4 * kMaxLen];
    float2 tw32[4 * kMaxLen];
    double s2[4 * kMaxLen];
    Tables tb{};
    const double two_pi = 6.283185307179586476925286766559;
    const double pi = 3.14159265358979323846264338327950;
    double2* dtw64 = reinterpret_cast<double2*>(base + kTablesOff);
    float2* dtw32 = reinterpret_cast<float2*>(base + kTablesOff + kTw64Bytes);
    double* ds2 = reinterpret_cast<double*>(base + kTablesOff + kTw64Bytes + kTw32Bytes);
    int off = 0;
    for (int mu = 0; mu < 4; mu++) {
        const int L = dims[mu];
        double mx = 0;
        for (int m = 0; m < L; m++) {
            const double a = two_pi * m / L;
            tw64[off + m] = make_double2(cos(a), -sin(a));
            tw32[off + m] = make_float2((float)cos(a), (float)-sin(a));
            const double sv = sin(pi * m / L);
            s2[off + m] = 4.0 * sv * sv;
            if (s2[off + m] > mx) mx = s2[off + m];
        }
        tb.p2max += mx;
        tb.tw64[mu] = dtw64 + off;
        tb.tw32[mu] = dtw32 + off;
        tb.s2[mu] = ds2 + off;
        off += L;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    double2* Fd = reinterpret_cast<double2*>(base);
    Ctl* ctl = reinterpret_cast<Ctl*>(base + kCtlOff);
    double* m64 = reinterpret_cast<double*>(base + kMultOff);
    float* m32 = reinterpret_cast<float*>(base + kMultOff + (size_t)kMaxSites * sizeof(double));
    if (cudaMemcpyAsync(dtw64, tw64, off * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dtw32, tw32, off * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ds2, s2, off * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess)
        return LGF_ERR_CUDA;
    launch_make_mult(s, d, tb, m64, m32);  // the accelerator's multiplier per momentum
    tb.mult64 = m64;
    tb.mult32 = m32;
    launch_pack_delta(s, d.V, Delta_in, Fd);
    launch_xy_fft<double>(d, sh, tb, s, Fd, false);
    launch_zt<double>(d, sh, tb, s, Fd, ctl);
    launch_xy_fft<double>(d, sh, tb, s, Fd, true);
    launch_unpack_delta(s, d.V, Fd, Dt_out);
    if (cudaGetLastError() != cudaSuccess) return LGF_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LGF_ERR_CUDA;
    return LGF_OK;
}
