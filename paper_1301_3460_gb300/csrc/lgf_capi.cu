// C ABI of the gauge-fixing library (declarations and contracts in include/lgf.h).
//
// Host side: context and device memory, twiddle and momentum tables, kernel
// configuration, and the device-resident loop.  One lgf_fix is one CUDA graph
// launch: the iteration body sits in a conditional WHILE node whose condition
// the last kernel of the body sets from the device loop state, so the loop runs
// to convergence with no host round trip.  The mixed mode chains an FP32 loop,
// the FP64 re-projection and an FP64 loop inside the same graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/lgf.h"
#include "lgf_launch.h"

using namespace lgf;

namespace {

thread_local char g_last_error[256] = "";

void set_error(const char* what, cudaError_t e, const char* file, int line)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) {                               \
            set_error(#call, e_, __FILE__, __LINE__);          \
            return LGF_ERR_CUDA;                               \
        }                                                      \
    } while (0)

#define CKR(call)                        \
    do {                                 \
        int r_ = (call);                 \
        if (r_ != LGF_OK) return r_;     \
    } while (0)

constexpr int kHistCap = 65536;
constexpr int kRefreshEvery = 25;
// The 8-real form's rebuild divides by n2 = |u01|^2 + |u02|^2, so it holds a link
// to about 1e-15 / n2; among the 4 million links of a random 32^4 field the
// smallest n2 is ~5e-4, so 1e-10 accepts such fields and refuses links within
// n2 ~ 1e-5 of the form's singular set.
constexpr double kForm8Tol = 1e-10;
// FP32 phase: iterations without a new smallest theta before FP64 takes over.
// Far from FP32's floor (theta ~1e-14..1e-13 on 32^4) a long window, because the
// method's theta is not monotone (FP64 runs on Wilson-action configurations go up
// to ~1200 iterations between new minima); near it a short one.
constexpr int kStallIters = 2000;
constexpr int kStallNearIters = 50;
constexpr double kNearFloor = 1e-12;

bool length_ok(int L)
{
    return L == 4 || L == 6 || L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64 ||
           L == 96 || L == 128;
}

}  // namespace

struct lgf_ctx {
    int L[4] = {0, 0, 0, 0};
    int V = 0;
    int flags = 0;
    bool mixed = false, track = true;
    bool plain = false;  // steepest descent without Fourier acceleration
    cudaStream_t stream = nullptr;   // user stream for launches
    cudaStream_t cap = nullptr;      // private stream used to capture graphs
    Lat lat{};    // FP64 kernels (links with ne = 6 or 9 entries)
    Lat lat32{};  // FP32 kernels (always 6: rows 0,1)
    Shape sh64{}, sh32{};
    Tables tb{};
    // state
    double2* U64 = nullptr;
    double2* G64 = nullptr;
    double2* g64 = nullptr;   // [9][V]; also the FP64 reprojection of G at the precision switch
    float2* U32 = nullptr;    // FP32 links of the FP32 phase, and the second buffer the fused
    float2* U32b = nullptr;   // update writes (the two swap roles every update)
    float2* G32 = nullptr;
    float2* g32 = nullptr;
    float2* AH32 = nullptr;   // FP32 phase without the fused update: packed anti-Hermitian
    float* Fs32 = nullptr;    // parts and Re Tr handed from the update to the Delta kernel
    bool fused32 = false;     // FP32 phase: update fused with Delta (links recomputed) or not
    bool accel32 = false;     // FP64 iterations take the accelerator's transforms in FP32
    bool gu32 = false;        // FP32 phase: g builder and update in one persistent launch
    unsigned* gu_sync = nullptr;  // its queue, epoch and per-plane flags
    void* Fd = nullptr;       // [4][V] double2 (the FP32 phase uses the front half as float2)
    double2* AH64 = nullptr;  // [4][4][V] packed anti-Hermitian parts of the links
    double* Fs64 = nullptr;   // [V] Re Tr of the four links of a site
    double* partials = nullptr;
    Ctl* ctl = nullptr;       // loop state of lgf_fix
    Ctl* ctl_stage = nullptr; // state used by the stage entry points
    double2* hist = nullptr;
    unsigned long long* err = nullptr;
    double* stage = nullptr;  // device staging for host arrays
    size_t stage_bytes = 0;
    void* tables = nullptr;
    void* mult = nullptr;     // multiplier tables: V doubles then V floats
    Ctl* host_ctl = nullptr;  // pinned
    bool have_links = false;
    double switch_tol = 1e-6;
    int refresh_every = kRefreshEvery;  // FP32 phase: rebuild U32 from U_in and G every this many updates (0: never)
    unsigned int loop_bound = 0;  // test hook: cap on loop-body runs
    cudaGraphExec_t exec = nullptr;
    int last_iters = 0, last_iters32 = 0, last_hist = 0;
    // workspace of the derivative entry points (allocated on first use)
    double2* dGp = nullptr;   // [4][9][V] cotangent in / out
    double2* dGud = nullptr;  // [4][9][V]
    double2* dQ = nullptr;    // [4][9][V]
    double2* dGgs = nullptr;  // [6][V]
    double2* dFA = nullptr;   // [4][V]
    double2* dFB = nullptr;   // [4][V]
    double2* gl_part = nullptr;
    double2* gl_At = nullptr;  // [16][9]
    double* gl_D = nullptr;    // [5]
    double* wil_part = nullptr;  // plaquette partial sums, then the result
    int gen_precision = 64;      // arithmetic of the configuration generator's staples and draws
    float2* gen32 = nullptr;     // [4][6][V]: FP32 copy of the links for the FP32 generator's staples
};

namespace {

// Shared-memory FFT tiles: the four fields of an xy-plane, and one z,t pencil of
// xw x-columns; thread counts a multiple of 32 up to 128 (FP64) or 256 (FP32).
// zt_form 1: the persistent z,t kernel with TMA-staged pencils (its grid from
// the device's occupancy, so only with a GPU present).
bool make_shape(const Lat& d, size_t elem, int nt_xy, int nt_zt, int xw, Shape* sh, int zt_form = 0)
{
    const int ntmax = elem == sizeof(double2) ? 128 : 256;  // the tile kernels' launch bounds
    if (nt_xy < 32 || nt_xy > ntmax || nt_xy % 32 || nt_zt < 32 || nt_zt > ntmax || nt_zt % 32) return false;
    if (plane_tile_bytes(d, elem) > kTileBudget) return false;
    if (xw < 1 || (xw & (xw - 1)) || d.L[0] % xw) return false;  // a power of two dividing Lx
    if (pencil_tile_bytes(d, xw, elem) > kTileBudget) return false;
    if (zt_form < 0 || zt_form > 1) return false;
    int grid = 0;
    if (zt_form == 1) {
        grid = elem == sizeof(double2) ? zt_tma_grid<double>(d, nt_zt, xw) : zt_tma_grid<float>(d, nt_zt, xw);
        if (grid <= 0) return false;
    }
    sh->nt_xy = nt_xy;
    sh->nt_zt = nt_zt;
    sh->xw = xw;
    sh->zt_tma = zt_form;
    sh->zt_grid = grid;
    return true;
}

// default shape: the widest pencil up to the preferred width that fits
bool pick_shape(const Lat& d, size_t elem, int prefer_xw, Shape* sh)
{
    for (int xw = prefer_xw; xw >= 1; xw >>= 1)
        if (make_shape(d, elem, 128, 128, xw, sh)) return true;
    return false;
}


template <typename T> const Lat& lat_of(const lgf_ctx* c);
template <> const Lat& lat_of<double>(const lgf_ctx* c) { return c->lat; }
template <> const Lat& lat_of<float>(const lgf_ctx* c) { return c->lat32; }

template <typename T> const Shape& shape_of(const lgf_ctx* c);
template <> const Shape& shape_of<double>(const lgf_ctx* c) { return c->sh64; }
template <> const Shape& shape_of<float>(const lgf_ctx* c) { return c->sh32; }

// one FP64 iteration after Delta: FFT(z,t)+scale+IFFT(t,z), IFFT(x,y)+g, update,
// Delta+FFT(x,y)
// Delta, theta and F of the FP64 links with the forward x,y transform: in FP64, or
// in FP32 into the front half of Fd when the accelerator runs in FP32
void launch_delta64(lgf_ctx* c, cudaStream_t s, Ctl* ctl, double2* hist)
{
    if (c->accel32 && !c->plain)
        launch_delta64_f32(c->lat, c->sh64, s, c->AH64, c->Fs64, reinterpret_cast<float2*>(c->Fd), c->partials, ctl,
                           hist);
    else
        launch_delta<double>(c->lat, c->sh64, c->tb, s, c->AH64, c->Fs64, reinterpret_cast<double2*>(c->Fd),
                             c->partials, ctl, hist, !c->plain);
}

// the accelerator and the g builder of an FP64 iteration: FP64 transforms, or FP32
// transforms (z,t kernel of the FP32 phase, FP32 inverse x,y with the FP64
// Gram-Schmidt writing the FP64 g)
void launch_accel_g64(lgf_ctx* c, cudaStream_t s, Ctl* ctl)
{
    double2* Fd = reinterpret_cast<double2*>(c->Fd);
    if (c->accel32) {
        float2* Fd32 = reinterpret_cast<float2*>(c->Fd);
        launch_zt<float>(c->lat32, c->sh32, c->tb, s, Fd32, ctl);
        launch_xyinv_g32_64(c->lat32, c->sh32, s, Fd32, c->g64, ctl);
    } else {
        launch_zt<double>(c->lat, c->sh64, c->tb, s, Fd, ctl);
        launch_xyinv_g<double>(c->lat, c->sh64, c->tb, s, Fd, c->g64, ctl);
    }
}

void launch_body64(lgf_ctx* c, cudaStream_t s, double2* G)
{
    double2* Fd = reinterpret_cast<double2*>(c->Fd);
    const Lat& d = c->lat;
    if (c->plain)
        launch_build_g<double>(d, s, Fd, c->g64, c->ctl);
    else
        launch_accel_g64(c, s, c->ctl);
    launch_update<double>(d, s, c->U64, G, c->g64, c->ctl, c->AH64, c->Fs64);
    launch_delta64(c, s, c->ctl, c->hist);
}

// one FP32-phase iteration after Delta: FFT(z,t)+scale+IFFT(t,z), IFFT(x,y)+g, then
// either (fused) the update fused with Delta, theta and F, links src -> dst, on
// refresh iterations the FP32 links rebuilt from the input and Delta taken again,
// and FFT(x,y); or the update in place writing the links' packed anti-Hermitian
// parts, the refresh, and Delta+FFT(x,y)
void launch_body32(lgf_ctx* c, cudaStream_t s, const float2* src, float2* dst)
{
    float2* Fd = reinterpret_cast<float2*>(c->Fd);
    const Lat& d = c->lat32;
    if (c->plain) {
        launch_build_g<float>(d, s, Fd, c->g32, c->ctl);
    } else {
        launch_zt<float>(d, c->sh32, c->tb, s, Fd, c->ctl);
        if (!c->gu32 || c->fused32) launch_xyinv_g<float>(d, c->sh32, c->tb, s, Fd, c->g32, c->ctl);
    }
    if (c->fused32) {
        launch_update_delta32(d, s, src, dst, c->G32, c->g32, c->ctl, Fd, c->partials, c->hist);
        if (c->refresh_every > 0) {
            launch_refresh32(s, d, c->lat.ne, c->U64, c->G32, dst, nullptr, nullptr, c->ctl, c->refresh_every);
            launch_delta_links32(d, s, dst, Fd, c->partials, c->ctl, c->hist, c->refresh_every);
        }
        if (!c->plain) launch_xy_fft<float>(d, c->sh32, c->tb, s, Fd, false);
    } else {
        if (c->gu32 && !c->plain)
            launch_gu32(d, c->sh32, s, Fd, c->g32, c->U32, c->G32, c->AH32, c->Fs32, c->ctl, c->gu_sync);
        else
            launch_update<float>(d, s, c->U32, c->G32, c->g32, c->ctl, c->AH32, c->Fs32);
        if (c->refresh_every > 0)
            launch_refresh32(s, d, c->lat.ne, c->U64, c->G32, c->U32, c->AH32, c->Fs32, c->ctl, c->refresh_every);
        launch_delta<float>(d, c->sh32, c->tb, s, c->AH32, c->Fs32, Fd, c->partials, c->ctl, c->hist, !c->plain);
    }
}

// Delta, theta and F of the FP32 phase's first links (U32), transformed along x,y
void launch_start32(lgf_ctx* c, cudaStream_t s, Ctl* ctl, double2* hist)
{
    float2* Fd = reinterpret_cast<float2*>(c->Fd);
    if (c->fused32) {
        launch_delta_links32(c->lat32, s, c->U32, Fd, c->partials, ctl, hist, 0);
        if (!c->plain) launch_xy_fft<float>(c->lat32, c->sh32, c->tb, s, Fd, false);
    } else {
        launch_ah_init<float>(c->lat32, s, c->U32, c->AH32, c->Fs32);
        launch_delta<float>(c->lat32, c->sh32, c->tb, s, c->AH32, c->Fs32, Fd, c->partials, ctl, hist, !c->plain);
    }
}

// ---------------------------------------------------------------- graph

int capture_begin(lgf_ctx* c, cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps)
{
    CK(cudaStreamBeginCaptureToGraph(c->cap, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                     cudaStreamCaptureModeThreadLocal));
    return LGF_OK;
}

int capture_end(lgf_ctx* c, std::vector<cudaGraphNode_t>& deps)
{
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    CK(cudaGetLastError());
    CK(cudaStreamGetCaptureInfo(c->cap, &st, nullptr, nullptr, &d, nullptr, &nd));
    deps.assign(d, d + nd);
    cudaGraph_t out;
    CK(cudaStreamEndCapture(c->cap, &out));
    return LGF_OK;
}

// adds a WHILE node after deps; *body receives its body graph, *h its handle
int add_while(cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps, cudaGraph_t* body, cudaGraphConditionalHandle* h)
{
    CK(cudaGraphConditionalHandleCreate(h, graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = *h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
    *body = p.conditional.phGraph_out[0];
    deps.assign(1, node);
    return LGF_OK;
}

// FP64 loop: one iteration per body run
int add_loop64(lgf_ctx* c, cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps, double2* G)
{
    cudaGraph_t body;
    cudaGraphConditionalHandle h;
    CKR(add_while(graph, deps, &body, &h));
    CK(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_body64(c, c->cap, G);
    launch_loop_ctl(c->cap, c->ctl, h);
    CK(cudaGetLastError());
    cudaGraph_t out;
    CK(cudaStreamEndCapture(c->cap, &out));
    return LGF_OK;
}

// FP32 loop: two iterations per body run, links U32 -> U32b -> U32 when the update
// is fused with Delta, so that the two link buffers keep fixed roles in the graph
// (when the first iteration ends the phase, every kernel of the second returns at
// once); in place in U32 otherwise
int add_loop32(lgf_ctx* c, cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps)
{
    cudaGraph_t body;
    cudaGraphConditionalHandle h;
    CKR(add_while(graph, deps, &body, &h));
    CK(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_body32(c, c->cap, c->U32, c->fused32 ? c->U32b : c->U32);
    launch_body32(c, c->cap, c->fused32 ? c->U32b : c->U32, c->U32);
    launch_loop_ctl(c->cap, c->ctl, h);
    CK(cudaGetLastError());
    cudaGraph_t out;
    CK(cudaStreamEndCapture(c->cap, &out));
    return LGF_OK;
}

// Append the nodes of one lgf_fix of context c to graph after deps; deps
// receives the terminal node.
int append_fix(lgf_ctx* c, cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps)
{
    if (c->mixed) {
        CKR(capture_begin(c, graph, deps));
        launch_mixed_prep(c->cap, c->V, c->lat.ne, c->U64, c->U32, c->G32, c->ctl);
        launch_start32(c, c->cap, c->ctl, c->hist);
        CKR(capture_end(c, deps));
        CKR(add_loop32(c, graph, deps));
        CKR(capture_begin(c, graph, deps));
        launch_switch(c->cap, c->lat, c->G32, c->g64, c->U64, c->G64, c->ctl);
        launch_ah_init<double>(c->lat, c->cap, c->U64, c->AH64, c->Fs64);
        launch_delta64(c, c->cap, c->ctl, c->hist);
        CKR(capture_end(c, deps));
        CKR(add_loop64(c, graph, deps, c->G64));
    } else {
        CKR(capture_begin(c, graph, deps));
        launch_ah_init<double>(c->lat, c->cap, c->U64, c->AH64, c->Fs64);
        launch_delta64(c, c->cap, c->ctl, c->hist);
        CKR(capture_end(c, deps));
        CKR(add_loop64(c, graph, deps, c->track ? c->G64 : nullptr));
    }
    return LGF_OK;
}

int instantiate(cudaGraph_t graph, cudaGraphExec_t* exec)
{
    cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        set_error("cudaGraphInstantiate", e, __FILE__, __LINE__);
        *exec = nullptr;
        return LGF_ERR_CUDA;
    }
    return LGF_OK;
}

int build_graph(lgf_ctx* c)
{
    if (c->exec) return LGF_OK;
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    std::vector<cudaGraphNode_t> deps;
    int r = append_fix(c, graph, deps);
    if (r != LGF_OK) {
        cudaGraphDestroy(graph);
        return r;
    }
    return instantiate(graph, &c->exec);
}

void drop_graph(lgf_ctx* c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;
}

// ---------------------------------------------------------------- set-up

int alloc(void** p, size_t bytes)
{
    CK(cudaMalloc(p, bytes));
    return LGF_OK;
}

int ensure_stage(lgf_ctx* c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return LGF_OK;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    CKR(alloc((void**)&c->stage, bytes));
    c->stage_bytes = bytes;
    return LGF_OK;
}

int build_tables(lgf_ctx* c)
{
    size_t n = 0;
    for (int mu = 0; mu < 4; mu++) n += c->L[mu];
    const size_t bytes = n * (sizeof(double2) + sizeof(float2) + sizeof(double) + sizeof(float));
    CKR(alloc(&c->tables, bytes));
    std::vector<unsigned char> h(bytes);
    double2* t64 = reinterpret_cast<double2*>(h.data());
    float2* t32 = reinterpret_cast<float2*>(h.data() + n * sizeof(double2));
    double* s2 = reinterpret_cast<double*>(h.data() + n * (sizeof(double2) + sizeof(float2)));
    float* s2f = reinterpret_cast<float*>(h.data() + n * (sizeof(double2) + sizeof(float2) + sizeof(double)));
    const double two_pi = 6.283185307179586476925286766559;
    const double pi = 3.14159265358979323846264338327950;
    size_t off = 0;
    c->tb.p2max = 0;
    for (int mu = 0; mu < 4; mu++) {
        const int L = c->L[mu];
        double mx = 0;
        for (int m = 0; m < L; m++) {
            const double a = two_pi * m / L;
            t64[off + m] = make_double2(cos(a), -sin(a));  // exp(-2 pi i m / L)
            t32[off + m] = make_float2((float)cos(a), (float)-sin(a));
            const double sv = sin(pi * m / L);
            s2[off + m] = 4.0 * sv * sv;
            s2f[off + m] = (float)s2[off + m];
            if (s2[off + m] > mx) mx = s2[off + m];
        }
        c->tb.p2max += mx;
        unsigned char* base = reinterpret_cast<unsigned char*>(c->tables);
        c->tb.tw64[mu] = reinterpret_cast<const double2*>(base) + off;
        c->tb.tw32[mu] = reinterpret_cast<const float2*>(base + n * sizeof(double2)) + off;
        c->tb.s2[mu] = reinterpret_cast<const double*>(base + n * (sizeof(double2) + sizeof(float2))) + off;
        off += L;
    }
    c->tb.s2f = reinterpret_cast<const float*>(reinterpret_cast<unsigned char*>(c->tables) +
                                               n * (sizeof(double2) + sizeof(float2) + sizeof(double)));
    CK(cudaMemcpy(c->tables, h.data(), bytes, cudaMemcpyHostToDevice));
    // p2max/(p2(k) V) for every momentum, in both precisions
    const size_t Vs = (size_t)c->V;
    CKR(alloc(&c->mult, Vs * (sizeof(double) + sizeof(float))));
    double* m64 = reinterpret_cast<double*>(c->mult);
    float* m32 = reinterpret_cast<float*>(m64 + Vs);
    launch_make_mult(nullptr, c->lat, c->tb, m64, m32);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    c->tb.mult64 = m64;
    c->tb.mult32 = m32;
    return LGF_OK;
}

int create_impl(const int dims[4], int flags, lgf_ctx* c)
{
    for (int mu = 0; mu < 4; mu++) {
        if (!length_ok(dims[mu])) return LGF_ERR_UNSUPPORTED_DIMS;
        c->L[mu] = dims[mu];
    }
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * 24 > 0x7fffffffL) return LGF_ERR_UNSUPPORTED_DIMS;  // plane offsets are 32-bit
    c->V = (int)V;
    c->flags = flags;
    c->mixed = (flags & LGF_MIXED) != 0;
    c->plain = (flags & LGF_PLAIN_SD) != 0;
    c->track = c->mixed || !(flags & LGF_NO_GAUGE);
    Lat& d = c->lat;
    int st = 1;
    for (int mu = 0; mu < 4; mu++) {
        d.L[mu] = dims[mu];
        d.stride[mu] = st;
        st *= dims[mu];
    }
    d.V = c->V;
    d.P = dims[0] * dims[1];
    d.nplanes = dims[2] * dims[3];
    lat_set_divisors(d);
    d.ne = (flags & LGF_LINKS18) ? 9 : (flags & LGF_LINKS8) ? 4 : 6;
    c->lat32 = d;
    c->lat32.ne = 6;
    if (!pick_shape(d, sizeof(double2), 4, &c->sh64)) return LGF_ERR_UNSUPPORTED_DIMS;
    if (!pick_shape(d, sizeof(float2), 8, &c->sh32)) return LGF_ERR_UNSUPPORTED_DIMS;

    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (ndev < 1) return LGF_ERR_CUDA;
    CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    CK(prepare_kernels<double>(d, c->sh64));
    if (c->mixed) CK(prepare_kernels<float>(d, c->sh32));

    const size_t Vs = (size_t)c->V;
    CKR(alloc((void**)&c->U64, (size_t)4 * d.ne * Vs * sizeof(double2)));
    if (c->track) CKR(alloc((void**)&c->G64, 6 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->g64, 9 * Vs * sizeof(double2)));
    CKR(alloc(&c->Fd, 4 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->AH64, 16 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->Fs64, Vs * sizeof(double)));
    if (c->mixed) {
        CKR(alloc((void**)&c->U32, 24 * Vs * sizeof(float2)));
        CKR(alloc((void**)&c->U32b, 24 * Vs * sizeof(float2)));
        CKR(alloc((void**)&c->AH32, 16 * Vs * sizeof(float2)));
        CKR(alloc((void**)&c->Fs32, Vs * sizeof(float)));
        CKR(alloc((void**)&c->G32, 6 * Vs * sizeof(float2)));
        CKR(alloc((void**)&c->g32, 9 * Vs * sizeof(float2)));
        // the FP32 phase's default form: g builder and update in one persistent launch
        CK(gu32_prepare(c->lat32));
        CKR(alloc((void**)&c->gu_sync, (size_t)(4 + d.nplanes) * sizeof(unsigned)));
        CK(cudaMemset(c->gu_sync, 0, (size_t)(4 + d.nplanes) * sizeof(unsigned)));
        c->gu32 = true;
    }
    // block partial sums of theta and F: one pair per plane (Delta kernel) or per
    // block of the site-parallel kernels, whichever grid is larger
    const size_t nblk = (size_t)std::max(d.nplanes, update_grid(c->V));
    CKR(alloc((void**)&c->partials, 2 * nblk * sizeof(double)));
    CKR(alloc((void**)&c->ctl, sizeof(Ctl)));
    CKR(alloc((void**)&c->ctl_stage, sizeof(Ctl)));
    CKR(alloc((void**)&c->hist, kHistCap * sizeof(double2)));
    CKR(alloc((void**)&c->err, 3 * sizeof(unsigned long long)));
    CK(cudaMemset(c->ctl, 0, sizeof(Ctl)));
    CK(cudaMemset(c->ctl_stage, 0, sizeof(Ctl)));
    CK(cudaMallocHost((void**)&c->host_ctl, sizeof(Ctl)));
    CKR(build_tables(c));
    return LGF_OK;
}

void free_all(lgf_ctx* c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    void* ptrs[] = {c->U64, c->G64, c->g64, c->U32, c->G32, c->g32, c->Fd, c->partials, c->ctl, c->ctl_stage,
                    c->hist, c->err, c->stage, c->tables, c->mult, c->AH64, c->Fs64, c->U32b, c->AH32, c->Fs32, c->dGp, c->dGud, c->dQ, c->dGgs, c->dFA, c->dFB,
                    c->gl_part, c->gl_At, c->gl_D, c->wil_part, c->gen32, c->gu_sync};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->host_ctl) cudaFreeHost(c->host_ctl);
    if (c->cap) cudaStreamDestroy(c->cap);
}

// copy a caller array to device memory (or use it in place) and return the device pointer
// Device address of a page-locked (pinned or registered) host buffer, so that a
// kernel can read or write it in place over the host link; null for pageable
// memory.
const void* mapped_host(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

int stage_in(lgf_ctx* c, const double* p, size_t bytes, int on_device, const double** out)
{
    if (on_device) {
        *out = p;
        return LGF_OK;
    }
    if (const void* d = mapped_host(p)) {  // pinned host memory: the kernel reads it directly
        *out = static_cast<const double*>(d);
        return LGF_OK;
    }
    CKR(ensure_stage(c, bytes));
    CK(cudaMemcpyAsync(c->stage, p, bytes, cudaMemcpyHostToDevice, c->stream));
    *out = c->stage;
    return LGF_OK;
}

// *dev: where the kernel writes; *copy: whether stage_out_end must copy it to p.
// Host outputs always go through the device staging buffer and one copy: a
// kernel's scattered 144-byte records written straight into pinned host memory
// cross the host link seven times slower than one bulk copy.
int stage_out_begin(lgf_ctx* c, double* p, size_t bytes, int on_device, double** dev, bool* copy)
{
    *copy = false;
    if (on_device) {
        *dev = p;
        return LGF_OK;
    }
    CKR(ensure_stage(c, bytes));
    *dev = c->stage;
    *copy = true;
    return LGF_OK;
}

int stage_out_end(lgf_ctx* c, double* p, size_t bytes, bool copy)
{
    if (copy) CK(cudaMemcpyAsync(p, c->stage, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    return LGF_OK;
}

int reset_stage_ctl(lgf_ctx* c, double alpha = 0.0)
{
    Ctl h;
    memset(&h, 0, sizeof h);
    h.alpha = alpha;
    h.tol = -1.0;
    h.tol_final = -1.0;
    h.max_iter = 0x7fffffff;
    h.phase = 1;
    *c->host_ctl = h;
    CK(cudaMemcpyAsync(c->ctl_stage, c->host_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    return LGF_OK;
}

// LGF_ERR_TIMEOUT when a kernel of the last stage call gave up waiting for its own
// tensor copies (Ctl::fault of the stage state)
int stage_fault(lgf_ctx* c)
{
    CK(cudaMemcpyAsync(&c->host_ctl->fault, &c->ctl_stage->fault, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->host_ctl->fault) {
        set_error("a z,t kernel gave up waiting for its tensor copies", cudaSuccess, __FILE__, __LINE__);
        return LGF_ERR_TIMEOUT;
    }
    return LGF_OK;
}

// ---------------------------------------------------------------- autotuner

// Launch shapes of the plane-tiled kernels are chosen per lattice shape and
// precision by timing the candidates on the context's own data; the choice is
// kept for the process, so contexts of equal extents are tuned once.
std::mutex g_tune_mutex;
std::map<std::array<int, 5>, Shape> g_tuned;

template <typename T> Shape& shape_ref(lgf_ctx* c);
template <> Shape& shape_ref<double>(lgf_ctx* c) { return c->sh64; }
template <> Shape& shape_ref<float>(lgf_ctx* c) { return c->sh32; }

template <typename T> vec2_t<T>* g_of(lgf_ctx* c);
template <> double2* g_of<double>(lgf_ctx* c) { return c->g64; }
template <> float2* g_of<float>(lgf_ctx* c) { return c->g32; }

// mean time of `reps` launches of the xy kernels (which = 0) or the zt kernel (1)
template <typename T> int time_shape(lgf_ctx* c, const Shape& sh, int which, float* ms)
{
    const int reps = 3;
    cudaStream_t s = c->stream;
    vec2_t<T>* Fd = reinterpret_cast<vec2_t<T>*>(c->Fd);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int r = 0; r <= reps; r++) {
        if (r == 1) cudaEventRecord(e0, s);
        if (which == 0) {
            // the plane kernels of the precision's iteration: FP64 Delta + FFT(x,y) and
            // IFFT(x,y) + g; FP32 FFT(x,y) and IFFT(x,y) + g
            if constexpr (sizeof(T) == 8)
                launch_delta<double>(c->lat, sh, c->tb, s, c->AH64, c->Fs64, reinterpret_cast<double2*>(c->Fd),
                                     c->partials, c->ctl_stage, nullptr, true);
            else if (c->fused32)
                launch_xy_fft<float>(c->lat32, sh, c->tb, s, reinterpret_cast<float2*>(c->Fd), false);
            else
                launch_delta<float>(c->lat32, sh, c->tb, s, c->AH32, c->Fs32, reinterpret_cast<float2*>(c->Fd),
                                    c->partials, c->ctl_stage, nullptr, true);
            launch_xyinv_g<T>(lat_of<T>(c), sh, c->tb, s, Fd, g_of<T>(c), c->ctl_stage);
        } else {
            launch_zt<T>(lat_of<T>(c), sh, c->tb, s, Fd, c->ctl_stage);
        }
    }
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_error("autotune timing", e, __FILE__, __LINE__);
        return LGF_ERR_CUDA;
    }
    CK(cudaGetLastError());
    *ms = t / reps;
    return LGF_OK;
}

template <typename T> int autotune_prec(lgf_ctx* c)
{
    const size_t elem = sizeof(vec2_t<T>);
    std::array<int, 5> key = {c->L[0], c->L[1], c->L[2], c->L[3], (int)elem};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            shape_ref<T>(c) = it->second;
            return LGF_OK;
        }
    }
    Shape best = shape_ref<T>(c);
    float best_xy = 1e30f, best_zt = 1e30f;
    const int nts[3] = {64, 128, 256};
    for (int nt : nts) {
        Shape cand;
        if (!make_shape(lat_of<T>(c), elem, nt, best.nt_zt, best.xw, &cand)) continue;
        float ms;
        CKR(time_shape<T>(c, cand, 0, &ms));
        if (ms < best_xy) {
            best_xy = ms;
            best.nt_xy = cand.nt_xy;
        }
    }
    for (int form = 0; form <= 1; form++)
        for (int nt : nts)
            for (int xw = 1; xw <= 16; xw <<= 1) {
                Shape cand;
                if (!make_shape(lat_of<T>(c), elem, best.nt_xy, nt, xw, &cand, form)) continue;
                float ms;
                CKR(time_shape<T>(c, cand, 1, &ms));
                if (ms < best_zt) {
                    best_zt = ms;
                    best.nt_zt = cand.nt_zt;
                    best.xw = cand.xw;
                    best.zt_tma = cand.zt_tma;
                    best.zt_grid = cand.zt_grid;
                }
            }
    shape_ref<T>(c) = best;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = best;
    return LGF_OK;
}

int autotune_ctx(lgf_ctx* c)
{
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(reset_stage_ctl(c, 0.08));
    launch_ah_init<double>(c->lat, c->stream, c->U64, c->AH64, c->Fs64);
    CKR(autotune_prec<double>(c));
    if (c->mixed) {
        launch_mixed_prep(c->stream, c->V, c->lat.ne, c->U64, c->U32, c->G32, c->ctl_stage);
        launch_start32(c, c->stream, c->ctl_stage, nullptr);
        CKR(autotune_prec<float>(c));
    }
    CK(cudaStreamSynchronize(c->stream));
    drop_graph(c);
    return LGF_OK;
}

int ensure_diff(lgf_ctx* c)
{
    if (c->dGp) return LGF_OK;
    const size_t Vs = (size_t)c->V;
    CKR(alloc((void**)&c->dGp, 36 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->dGud, 36 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->dQ, 36 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->dGgs, 6 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->dFA, 4 * Vs * sizeof(double2)));
    CKR(alloc((void**)&c->dFB, 4 * Vs * sizeof(double2)));
    return LGF_OK;
}

int ensure_plaq(lgf_ctx* c)
{
    if (c->wil_part) return LGF_OK;
    return alloc((void**)&c->wil_part, (size_t)(plaquette_blocks(c->V) + 1) * sizeof(double));
}

int ensure_gluon(lgf_ctx* c)
{
    if (c->gl_part) return LGF_OK;
    CKR(alloc((void**)&c->gl_part, (size_t)16 * gluon_blocks(c->V) * 9 * sizeof(double2)));
    CKR(alloc((void**)&c->gl_At, 144 * sizeof(double2)));
    CKR(alloc((void**)&c->gl_D, 5 * sizeof(double)));
    return LGF_OK;
}

}  // namespace

// ---------------------------------------------------------------- batch

struct lgf_batch {
    std::vector<lgf_ctx*> ctx;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long* stamps = nullptr;  // device: [0] start, [1 + i] retirement of configuration i
    std::vector<unsigned long long> host_stamps;
    double* stage = nullptr;
    size_t stage_bytes = 0;
    bool tuned = false;
};

namespace {

void batch_free(lgf_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (lgf_ctx* c : b->ctx) {
        if (c) {
            free_all(c);
            delete c;
        }
    }
    if (b->stamps) cudaFree(b->stamps);
    if (b->stage) cudaFree(b->stage);
}

int batch_build(lgf_batch* b)
{
    if (b->exec) return LGF_OK;
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    std::vector<cudaGraphNode_t> root;
    lgf_ctx* c0 = b->ctx[0];
    int r = capture_begin(c0, graph, root);
    if (r == LGF_OK) {
        launch_stamp(c0->cap, b->stamps);
        r = capture_end(c0, root);
    }
    for (size_t i = 0; i < b->ctx.size() && r == LGF_OK; i++) {
        std::vector<cudaGraphNode_t> deps = root;  // every configuration is an independent branch
        r = append_fix(b->ctx[i], graph, deps);
        if (r == LGF_OK) r = capture_begin(b->ctx[i], graph, deps);
        if (r == LGF_OK) {
            launch_stamp(b->ctx[i]->cap, b->stamps + 1 + i);
            r = capture_end(b->ctx[i], deps);
        }
    }
    if (r != LGF_OK) {
        cudaGraphDestroy(graph);
        return r;
    }
    return instantiate(graph, &b->exec);
}

Ctl initial_ctl(const lgf_ctx* c, double alpha, double tol, int max_iter)
{
    Ctl h;
    memset(&h, 0, sizeof h);
    h.tol_final = tol;
    h.tol = c->mixed ? (c->switch_tol > tol ? c->switch_tol : tol) : tol;
    h.alpha = alpha;
    h.max_iter = max_iter;
    h.phase = c->mixed ? 0 : 1;
    h.hist_cap = kHistCap;
    h.loop_bound = c->loop_bound;
    h.theta_best = 1.0e300;
    h.iter_best = 0;
    h.stall = c->mixed ? kStallIters : 0;
    h.stall_near = kStallNearIters;
    h.near_floor = kNearFloor;
    return h;
}

int status_of(const Ctl& r)
{
    if (r.fault) {
        set_error("a z,t kernel gave up waiting for its tensor copies", cudaSuccess, __FILE__, __LINE__);
        return LGF_ERR_TIMEOUT;
    }
    if (r.nan_seen) return LGF_ERR_NAN;
    if (r.converged) return LGF_OK;
    if (!r.done) return LGF_ERR_TIMEOUT;
    return LGF_ERR_NOT_CONVERGED;
}

}  // namespace

// ==================================================================== C ABI

extern "C" {

const char* lgf_strerror(int status)
{
    switch (status) {
    case LGF_OK: return "ok";
    case LGF_ERR_ARG: return "invalid argument";
    case LGF_ERR_CUDA: return "CUDA error";
    case LGF_ERR_NOT_SU3: return "input links are not SU(3) to 1e-12";
    case LGF_ERR_UNSUPPORTED_DIMS: return "unsupported lattice extents";
    case LGF_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case LGF_ERR_NAN: return "theta or F became NaN or infinite";
    case LGF_ERR_TIMEOUT: return "device loop hit its safety bound, or a kernel timed out on its own copies";
    case LGF_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

const char* lgf_last_error(void) { return g_last_error; }

int lgf_create(const int dims[4], int flags, lgf_ctx** out)
{
    if (!dims || !out) return LGF_ERR_ARG;
    *out = nullptr;
    if (flags & ~(LGF_MIXED | LGF_NO_GAUGE | LGF_PLAIN_SD | LGF_LINKS18 | LGF_LINKS8)) return LGF_ERR_ARG;
    if ((flags & LGF_LINKS18) && (flags & LGF_LINKS8)) return LGF_ERR_ARG;
    lgf_ctx* c = new (std::nothrow) lgf_ctx();
    if (!c) return LGF_ERR_ARG;
    int r = create_impl(dims, flags, c);
    if (r != LGF_OK) {
        free_all(c);
        delete c;
        return r;
    }
    *out = c;
    return LGF_OK;
}

void lgf_destroy(lgf_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

int lgf_set_stream(lgf_ctx* c, void* stream)
{
    if (!c) return LGF_ERR_ARG;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    return LGF_OK;
}

int lgf_set_loop_bound(lgf_ctx* c, int max_body_runs)
{
    if (!c || max_body_runs < 0) return LGF_ERR_ARG;
    c->loop_bound = (unsigned int)max_body_runs;
    return LGF_OK;
}

int lgf_set_switch_tol(lgf_ctx* c, double tol)
{
    if (!c || !(tol >= 0)) return LGF_ERR_ARG;
    c->switch_tol = tol;
    return LGF_OK;
}

int lgf_set_fp32_refresh(lgf_ctx* c, int every)
{
    if (!c || every < 0) return LGF_ERR_ARG;
    if (every != c->refresh_every) {
        c->refresh_every = every;
        drop_graph(c);  // the interval is a launch argument of the captured body
    }
    return LGF_OK;
}

int lgf_set_accel_precision(lgf_ctx* c, int precision)
{
    if (!c || (precision != 64 && precision != 32)) return LGF_ERR_ARG;
    if (!c->mixed || c->plain) return LGF_ERR_STATE;
    const bool on = precision == 32;
    if (on) CK(prepare_accel32(c->lat));
    if (c->accel32 != on) {
        CK(cudaStreamSynchronize(c->stream));
        c->accel32 = on;
        drop_graph(c);
    }
    return LGF_OK;
}

int lgf_set_fp32_update(lgf_ctx* c, int form)
{
    if (!c || form < 0 || form > 2) return LGF_ERR_ARG;
    if (form == 2) {
        if (!c->mixed) return LGF_ERR_STATE;
        if (!c->gu_sync) {
            CK(gu32_prepare(c->lat32));
            CKR(alloc((void**)&c->gu_sync, (size_t)(4 + c->lat32.nplanes) * sizeof(unsigned)));
            CK(cudaMemsetAsync(c->gu_sync, 0, (size_t)(4 + c->lat32.nplanes) * sizeof(unsigned), c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    }
    if (c->fused32 != (form == 1) || c->gu32 != (form == 2)) {
        c->fused32 = form == 1;
        c->gu32 = form == 2;
        drop_graph(c);
    }
    return LGF_OK;
}

int lgf_set_links(lgf_ctx* c, const double* U, int on_device)
{
    if (!c || !U) return LGF_ERR_ARG;
    const size_t bytes = (size_t)4 * c->V * 18 * sizeof(double);
    const double* src;
    c->have_links = false;
    CKR(stage_in(c, U, bytes, on_device, &src));
    CK(cudaMemsetAsync(c->err, 0, 3 * sizeof(unsigned long long), c->stream));
    launch_pack_links64(c->stream, c->V, c->lat.ne, src, c->U64, c->err);
    if (c->track) launch_identity_rows64(c->stream, c->V, c->G64);
    CK(cudaGetLastError());
    unsigned long long e[3];
    CK(cudaMemcpyAsync(e, c->err, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double eu, ed, ef;
    memcpy(&eu, &e[0], sizeof eu);
    memcpy(&ed, &e[1], sizeof ed);
    memcpy(&ef, &e[2], sizeof ef);
    if (!(eu < 1e-12) || !(ed < 1e-12)) return LGF_ERR_NOT_SU3;
    if (!(ef < kForm8Tol)) return LGF_ERR_NOT_SU3;  // 8-real form only (0 otherwise)
    c->have_links = true;
    return LGF_OK;
}

int lgf_fix(lgf_ctx* c, double alpha, double theta_tol, int max_iter, int* iters, double* F, double* theta)
{
    if (!c) return LGF_ERR_ARG;
    if (!(alpha > 0) || !(theta_tol >= 0) || max_iter < 0) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(build_graph(c));
    *c->host_ctl = initial_ctl(c, alpha, theta_tol, max_iter);
    CK(cudaMemcpyAsync(c->ctl, c->host_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    CK(cudaGraphLaunch(c->exec, c->stream));
    CK(cudaMemcpyAsync(c->host_ctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    const Ctl r = *c->host_ctl;
    c->last_iters = r.iter;
    c->last_iters32 = r.iter_phase0;
    c->last_hist = r.iter + 1;
    if (iters) *iters = r.iter;
    if (F) *F = r.F;
    if (theta) *theta = r.theta;
    return status_of(r);
}

int lgf_get_links(lgf_ctx* c, double* U_out, int on_device)
{
    if (!c || !U_out) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    const size_t bytes = (size_t)4 * c->V * 18 * sizeof(double);
    double* dst;
    bool copy;
    CKR(stage_out_begin(c, U_out, bytes, on_device, &dst, &copy));
    launch_unpack_su3_64(c->stream, c->V, 4, c->lat.ne, c->U64, dst);
    CK(cudaGetLastError());
    return stage_out_end(c, U_out, bytes, copy);
}

int lgf_get_gauge(lgf_ctx* c, double* G_out, int on_device)
{
    if (!c || !G_out) return LGF_ERR_ARG;
    if (!c->track) return LGF_ERR_STATE;
    if (!c->have_links) return LGF_ERR_STATE;
    const size_t bytes = (size_t)c->V * 18 * sizeof(double);
    double* dst;
    bool copy;
    CKR(stage_out_begin(c, G_out, bytes, on_device, &dst, &copy));
    launch_unpack_su3_64(c->stream, c->V, 1, 6, c->G64, dst);
    CK(cudaGetLastError());
    return stage_out_end(c, G_out, bytes, copy);
}

int lgf_get_history(lgf_ctx* c, double* theta_F, int n_max, int* written)
{
    if (!c || !theta_F || n_max < 0) return LGF_ERR_ARG;
    int n = c->last_hist < kHistCap ? c->last_hist : kHistCap;
    if (n > n_max) n = n_max;
    if (n > 0) {
        CK(cudaMemcpyAsync(theta_F, c->hist, (size_t)n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (written) *written = n;
    return LGF_OK;
}

size_t lgf_links_state_bytes(const lgf_ctx* c)
{
    return c ? (size_t)4 * c->lat.ne * c->V * sizeof(double2) : 0;
}

int lgf_save_links(lgf_ctx* c, void* dst)
{
    if (!c || !dst) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CK(cudaMemcpyAsync(dst, c->U64, lgf_links_state_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LGF_OK;
}

int lgf_load_links(lgf_ctx* c, const void* src)
{
    if (!c || !src) return LGF_ERR_ARG;
    CK(cudaMemcpyAsync(c->U64, src, lgf_links_state_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    if (c->track) launch_identity_rows64(c->stream, c->V, c->G64);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    c->have_links = true;
    return LGF_OK;
}

int lgf_get_stats(lgf_ctx* c, int* iters_fp32, int* iters_fp64)
{
    if (!c) return LGF_ERR_ARG;
    if (iters_fp32) *iters_fp32 = c->last_iters32;
    if (iters_fp64) *iters_fp64 = c->last_iters - c->last_iters32;
    return LGF_OK;
}

int lgf_delta(lgf_ctx* c, double* Delta_out, int on_device, double* theta, double* F)
{
    if (!c) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(reset_stage_ctl(c));
    double2* Fd = reinterpret_cast<double2*>(c->Fd);
    launch_ah_init<double>(c->lat, c->stream, c->U64, c->AH64, c->Fs64);
    launch_delta<double>(c->lat, c->sh64, c->tb, c->stream, c->AH64, c->Fs64, Fd, c->partials, c->ctl_stage, nullptr,
                         false);
    CK(cudaGetLastError());
    if (Delta_out) {
        const size_t bytes = (size_t)c->V * 18 * sizeof(double);
        double* dst;
        bool copy;
        CKR(stage_out_begin(c, Delta_out, bytes, on_device, &dst, &copy));
        launch_unpack_delta(c->stream, c->V, Fd, dst);
        CK(cudaGetLastError());
        CKR(stage_out_end(c, Delta_out, bytes, copy));
    }
    CK(cudaMemcpyAsync(c->host_ctl, c->ctl_stage, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (theta) *theta = c->host_ctl->theta;
    if (F) *F = c->host_ctl->F;
    return LGF_OK;
}

int lgf_accelerate(lgf_ctx* c, const double* Delta_in, double* Dt_out, int on_device)
{
    if (!c || !Delta_in || !Dt_out) return LGF_ERR_ARG;
    const size_t bytes = (size_t)c->V * 18 * sizeof(double);
    const double* src;
    CKR(reset_stage_ctl(c));
    CKR(stage_in(c, Delta_in, bytes, on_device, &src));
    double2* Fd = reinterpret_cast<double2*>(c->Fd);
    launch_pack_delta(c->stream, c->V, src, Fd);
    launch_xy_fft<double>(c->lat, c->sh64, c->tb, c->stream, Fd, false);
    launch_zt<double>(c->lat, c->sh64, c->tb, c->stream, Fd, c->ctl_stage);
    launch_xy_fft<double>(c->lat, c->sh64, c->tb, c->stream, Fd, true);
    CK(cudaGetLastError());
    double* dst;
    bool copy;
    CKR(stage_out_begin(c, Dt_out, bytes, on_device, &dst, &copy));
    launch_unpack_delta(c->stream, c->V, Fd, dst);
    CK(cudaGetLastError());
    CKR(stage_out_end(c, Dt_out, bytes, copy));
    return stage_fault(c);
}

int lgf_build_g(lgf_ctx* c, const double* Dt_in, double alpha, double* g_out, int on_device)
{
    if (!c || !Dt_in || !g_out) return LGF_ERR_ARG;
    const size_t bytes = (size_t)c->V * 18 * sizeof(double);
    const double* src;
    // the forward x,y FFT below and the builder's inverse are both unnormalised, so the
    // builder sees Lx*Ly times the field: compensate in alpha, whose only use there is
    // the factor alpha/2 on the field
    CKR(reset_stage_ctl(c, alpha / (double)c->lat.P));
    CKR(stage_in(c, Dt_in, bytes, on_device, &src));
    double2* Fd = reinterpret_cast<double2*>(c->Fd);
    launch_pack_delta(c->stream, c->V, src, Fd);
    // the builder takes fields transformed along x and y: transform, then let it invert
    launch_xy_fft<double>(c->lat, c->sh64, c->tb, c->stream, Fd, false);
    launch_xyinv_g<double>(c->lat, c->sh64, c->tb, c->stream, Fd, c->g64, c->ctl_stage);
    CK(cudaGetLastError());
    double* dst;
    bool copy;
    CKR(stage_out_begin(c, g_out, bytes, on_device, &dst, &copy));
    launch_unpack_full(c->stream, c->V, c->g64, dst);
    CK(cudaGetLastError());
    return stage_out_end(c, g_out, bytes, copy);
}

// FP32-phase stage entry points: the FP32 phase's own kernels between FP64
// inputs and outputs.  The FP32 fields occupy the front half of Fd; results are
// widened into g64 ([9][V] double2) and unpacked from there.
int lgf_delta32(lgf_ctx* c, double* Delta_out, int on_device, double* theta, double* F)
{
    if (!c) return LGF_ERR_ARG;
    if (!c->mixed || !c->have_links) return LGF_ERR_STATE;
    CKR(reset_stage_ctl(c));
    float2* Fd32 = reinterpret_cast<float2*>(c->Fd);
    // the FP32 phase's start: links rounded to FP32, Delta, theta and F, the
    // forward x,y transform of Delta
    launch_mixed_prep(c->stream, c->V, c->lat.ne, c->U64, c->U32, c->G32, c->ctl_stage);
    launch_start32(c, c->stream, c->ctl_stage, nullptr);
    CK(cudaGetLastError());
    if (Delta_out) {
        double scale = 1.0;
        if (!c->plain) {  // back along x,y (unnormalised: P times the field)
            launch_xy_fft<float>(c->lat32, c->sh32, c->tb, c->stream, Fd32, true);
            scale = 1.0 / (double)c->lat.P;
        }
        launch_planes_to64(c->stream, 4L * c->V, Fd32, c->g64, scale);
        const size_t bytes = (size_t)c->V * 18 * sizeof(double);
        double* dst;
        bool copy;
        CKR(stage_out_begin(c, Delta_out, bytes, on_device, &dst, &copy));
        launch_unpack_delta(c->stream, c->V, c->g64, dst);
        CK(cudaGetLastError());
        CKR(stage_out_end(c, Delta_out, bytes, copy));
    }
    CK(cudaMemcpyAsync(c->host_ctl, c->ctl_stage, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (theta) *theta = c->host_ctl->theta;
    if (F) *F = c->host_ctl->F;
    return LGF_OK;
}

int lgf_accelerate32(lgf_ctx* c, const double* Delta_in, double* Dt_out, int on_device)
{
    if (!c || !Delta_in || !Dt_out) return LGF_ERR_ARG;
    if (!c->mixed) return LGF_ERR_STATE;
    const size_t bytes = (size_t)c->V * 18 * sizeof(double);
    const double* src;
    // the FP32 z,t kernel scales by (alpha/2) p2max/(p2 V): alpha = 2 gives the
    // accelerator itself
    CKR(reset_stage_ctl(c, 2.0));
    CKR(stage_in(c, Delta_in, bytes, on_device, &src));
    float2* Fd32 = reinterpret_cast<float2*>(c->Fd);
    launch_pack_delta(c->stream, c->V, src, c->g64);
    launch_planes_to32(c->stream, 4L * c->V, c->g64, Fd32, 1.0);
    launch_xy_fft<float>(c->lat32, c->sh32, c->tb, c->stream, Fd32, false);
    launch_zt<float>(c->lat32, c->sh32, c->tb, c->stream, Fd32, c->ctl_stage);
    launch_xy_fft<float>(c->lat32, c->sh32, c->tb, c->stream, Fd32, true);
    launch_planes_to64(c->stream, 4L * c->V, Fd32, c->g64, 1.0);
    CK(cudaGetLastError());
    double* dst;
    bool copy;
    CKR(stage_out_begin(c, Dt_out, bytes, on_device, &dst, &copy));
    launch_unpack_delta(c->stream, c->V, c->g64, dst);
    CK(cudaGetLastError());
    CKR(stage_out_end(c, Dt_out, bytes, copy));
    return stage_fault(c);
}

int lgf_build_g32(lgf_ctx* c, const double* Dt_in, double alpha, double* g_out, int on_device)
{
    if (!c || !Dt_in || !g_out) return LGF_ERR_ARG;
    if (!c->mixed) return LGF_ERR_STATE;
    const size_t bytes = (size_t)c->V * 18 * sizeof(double);
    const double* src;
    CKR(reset_stage_ctl(c, alpha));
    CKR(stage_in(c, Dt_in, bytes, on_device, &src));
    float2* Fd32 = reinterpret_cast<float2*>(c->Fd);
    // the FP32 builder takes fields transformed along x,y and already multiplied
    // by alpha/2, and its inverse x,y transform is unnormalised: rounded to FP32
    // times alpha/(2 P), then transformed forward
    launch_pack_delta(c->stream, c->V, src, c->g64);
    launch_planes_to32(c->stream, 4L * c->V, c->g64, Fd32, 0.5 * alpha / (double)c->lat.P);
    launch_xy_fft<float>(c->lat32, c->sh32, c->tb, c->stream, Fd32, false);
    launch_xyinv_g<float>(c->lat32, c->sh32, c->tb, c->stream, Fd32, c->g32, c->ctl_stage);
    launch_planes_to64(c->stream, 9L * c->V, c->g32, c->g64, 1.0);
    CK(cudaGetLastError());
    double* dst;
    bool copy;
    CKR(stage_out_begin(c, g_out, bytes, on_device, &dst, &copy));
    launch_unpack_full(c->stream, c->V, c->g64, dst);
    CK(cudaGetLastError());
    return stage_out_end(c, g_out, bytes, copy);
}

int lgf_time_kernels(lgf_ctx* c, double alpha, int n_iter, int precision, double* ms)
{
    if (!c || !ms || n_iter < 1 || !(alpha > 0)) return LGF_ERR_ARG;
    if (precision != 64 && precision != 32) return LGF_ERR_ARG;
    if (precision == 32 && !c->mixed) return LGF_ERR_STATE;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(reset_stage_ctl(c, alpha));
    cudaEvent_t ev[5];
    for (int i = 0; i < 5; i++) CK(cudaEventCreate(&ev[i]));
    std::vector<float> samples[4];
    cudaStream_t s = c->stream;
    int rc = LGF_OK;
    if (precision == 32) {
        launch_mixed_prep(s, c->V, c->lat.ne, c->U64, c->U32, c->G32, c->ctl_stage);
        launch_start32(c, s, c->ctl_stage, nullptr);
    } else {
        launch_ah_init<double>(c->lat, s, c->U64, c->AH64, c->Fs64);
    }
    for (int it = 0; it < n_iter && rc == LGF_OK; it++) {
        cudaEventRecord(ev[0], s);
        if (precision == 64) {
            // the kernels lgf_fix runs (the accelerator in FP32 when so set)
            double2* Fd = reinterpret_cast<double2*>(c->Fd);
            float2* Fd32 = reinterpret_cast<float2*>(c->Fd);
            if (c->accel32)
                launch_delta64_f32(c->lat, c->sh64, s, c->AH64, c->Fs64, Fd32, c->partials, c->ctl_stage, nullptr);
            else
                launch_delta<double>(c->lat, c->sh64, c->tb, s, c->AH64, c->Fs64, Fd, c->partials, c->ctl_stage,
                                     nullptr, true);
            cudaEventRecord(ev[1], s);
            if (c->accel32)
                launch_zt<float>(c->lat32, c->sh32, c->tb, s, Fd32, c->ctl_stage);
            else
                launch_zt<double>(c->lat, c->sh64, c->tb, s, Fd, c->ctl_stage);
            cudaEventRecord(ev[2], s);
            if (c->accel32)
                launch_xyinv_g32_64(c->lat32, c->sh32, s, Fd32, c->g64, c->ctl_stage);
            else
                launch_xyinv_g<double>(c->lat, c->sh64, c->tb, s, Fd, c->g64, c->ctl_stage);
            cudaEventRecord(ev[3], s);
            launch_update<double>(c->lat, s, c->U64, c->track ? c->G64 : nullptr, c->g64, c->ctl_stage, c->AH64,
                                  c->Fs64);
        } else {
            // FP32 phase.  Fused: FFT(x,y) alone, then z,t, IFFT(x,y) + g, and the update
            // fused with Delta, theta and F (links alternate between the two buffers).
            // Otherwise: Delta + FFT(x,y), z,t, IFFT(x,y) + g, the update.
            float2* Fd = reinterpret_cast<float2*>(c->Fd);
            if (c->fused32)
                launch_xy_fft<float>(c->lat32, c->sh32, c->tb, s, Fd, false);
            else
                launch_delta<float>(c->lat32, c->sh32, c->tb, s, c->AH32, c->Fs32, Fd, c->partials, c->ctl_stage,
                                    nullptr, true);
            cudaEventRecord(ev[1], s);
            launch_zt<float>(c->lat32, c->sh32, c->tb, s, Fd, c->ctl_stage);
            cudaEventRecord(ev[2], s);
            // the persistent g-and-update form: both in the g builder's slot, none in the update's
            if (c->gu32 && !c->fused32)
                launch_gu32(c->lat32, c->sh32, s, Fd, c->g32, c->U32, c->G32, c->AH32, c->Fs32, c->ctl_stage,
                            c->gu_sync);
            else
                launch_xyinv_g<float>(c->lat32, c->sh32, c->tb, s, Fd, c->g32, c->ctl_stage);
            cudaEventRecord(ev[3], s);
            if (c->fused32)
                launch_update_delta32(c->lat32, s, (it & 1) ? c->U32b : c->U32, (it & 1) ? c->U32 : c->U32b,
                                      c->G32, c->g32, c->ctl_stage, Fd, c->partials, nullptr);
            else if (!c->gu32)
                launch_update<float>(c->lat32, s, c->U32, c->G32, c->g32, c->ctl_stage, c->AH32, c->Fs32);
        }
        cudaEventRecord(ev[4], s);
        cudaError_t e = cudaEventSynchronize(ev[4]);
        if (e != cudaSuccess) {
            set_error("cudaEventSynchronize", e, __FILE__, __LINE__);
            rc = LGF_ERR_CUDA;
            break;
        }
        for (int k = 0; k < 4; k++) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            samples[k].push_back(t);
        }
    }
    for (int i = 0; i < 5; i++) cudaEventDestroy(ev[i]);
    if (rc != LGF_OK) return rc;
    CK(cudaGetLastError());
    // median over the iterations: a launch delayed by the host (the events bracket
    // the enqueue as well as the kernel) shows up as an outlier, not in the median
    for (int k = 0; k < 4; k++) {
        std::vector<float>& v = samples[k];
        std::sort(v.begin(), v.end());
        const size_t n = v.size();
        ms[k] = (n % 2) ? v[n / 2] : 0.5 * ((double)v[n / 2 - 1] + (double)v[n / 2]);
    }
    return LGF_OK;
}

int lgf_autotune(lgf_ctx* c)
{
    if (!c) return LGF_ERR_ARG;
    return autotune_ctx(c);
}

int lgf_set_shape(lgf_ctx* c, int precision, int nt_xy, int nt_zt, int xw, int zt_form)
{
    if (!c || (precision != 64 && precision != 32)) return LGF_ERR_ARG;
    if (precision == 32 && !c->mixed) return LGF_ERR_STATE;
    Shape sh;
    const bool ok = precision == 64 ? make_shape(c->lat, sizeof(double2), nt_xy, nt_zt, xw, &sh, zt_form)
                                    : make_shape(c->lat32, sizeof(float2), nt_xy, nt_zt, xw, &sh, zt_form);
    CK(cudaGetLastError());
    if (!ok) return LGF_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    (precision == 64 ? c->sh64 : c->sh32) = sh;
    drop_graph(c);
    return LGF_OK;
}

int lgf_get_shape(lgf_ctx* c, int precision, int* shape_out)
{
    if (!c || !shape_out || (precision != 64 && precision != 32)) return LGF_ERR_ARG;
    if (precision == 32 && !c->mixed) return LGF_ERR_STATE;
    const Shape& sh = precision == 64 ? c->sh64 : c->sh32;
    shape_out[0] = sh.nt_xy;
    shape_out[1] = sh.nt_zt;
    shape_out[2] = sh.xw;
    shape_out[3] = sh.zt_tma;
    shape_out[4] = sh.zt_grid;
    return LGF_OK;
}

int lgf_batch_create(int n, const int* dims, int flags, lgf_batch** out)
{
    if (n < 1 || !dims || !out) return LGF_ERR_ARG;
    *out = nullptr;
    if (flags & ~(LGF_MIXED | LGF_NO_GAUGE | LGF_PLAIN_SD | LGF_LINKS18 | LGF_LINKS8)) return LGF_ERR_ARG;
    if ((flags & LGF_LINKS18) && (flags & LGF_LINKS8)) return LGF_ERR_ARG;
    lgf_batch* b = new (std::nothrow) lgf_batch();
    if (!b) return LGF_ERR_ARG;
    int r = LGF_OK;
    for (int i = 0; i < n && r == LGF_OK; i++) {
        lgf_ctx* c = new (std::nothrow) lgf_ctx();
        if (!c) {
            r = LGF_ERR_ARG;
            break;
        }
        b->ctx.push_back(c);
        r = create_impl(dims + 4 * i, flags, c);
    }
    if (r == LGF_OK) {
        cudaError_t e = cudaMalloc((void**)&b->stamps, (n + 1) * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            set_error("cudaMalloc", e, __FILE__, __LINE__);
            r = LGF_ERR_CUDA;
        }
        b->host_stamps.assign(n + 1, 0ull);
    }
    if (r != LGF_OK) {
        batch_free(b);
        delete b;
        return r;
    }
    *out = b;
    return LGF_OK;
}

void lgf_batch_destroy(lgf_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

int lgf_batch_set_stream(lgf_batch* b, void* stream)
{
    if (!b) return LGF_ERR_ARG;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    for (lgf_ctx* c : b->ctx) c->stream = b->stream;
    return LGF_OK;
}

int lgf_batch_set_switch_tol(lgf_batch* b, double tol)
{
    if (!b || !(tol >= 0)) return LGF_ERR_ARG;
    for (lgf_ctx* c : b->ctx) c->switch_tol = tol;
    return LGF_OK;
}

int lgf_batch_set_fp32_update(lgf_batch* b, int form)
{
    if (!b) return LGF_ERR_ARG;
    CK(cudaStreamSynchronize(b->stream));
    for (lgf_ctx* c : b->ctx) CKR(lgf_set_fp32_update(c, form));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    return LGF_OK;
}

int lgf_batch_set_accel_precision(lgf_batch* b, int precision)
{
    if (!b) return LGF_ERR_ARG;
    for (lgf_ctx* c : b->ctx) CKR(lgf_set_accel_precision(c, precision));
    CK(cudaStreamSynchronize(b->stream));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    return LGF_OK;
}

int lgf_batch_set_links(lgf_batch* b, int i, const double* U, int on_device)
{
    if (!b || !U || i < 0 || i >= (int)b->ctx.size()) return LGF_ERR_ARG;
    lgf_ctx* c = b->ctx[i];
    if (on_device) return lgf_set_links(c, U, 1);
    if (mapped_host(U)) return lgf_set_links(c, U, 0);  // pinned: read in place
    // host arrays go through one staging buffer shared by the whole batch
    const size_t bytes = (size_t)4 * c->V * 18 * sizeof(double);
    if (b->stage_bytes < bytes) {
        if (b->stage) cudaFree(b->stage);
        b->stage = nullptr;
        b->stage_bytes = 0;
        CK(cudaMalloc((void**)&b->stage, bytes));
        b->stage_bytes = bytes;
    }
    CK(cudaMemcpyAsync(b->stage, U, bytes, cudaMemcpyHostToDevice, c->stream));
    return lgf_set_links(c, b->stage, 1);
}

int lgf_batch_fix(lgf_batch* b, double alpha, double theta_tol, int max_iter, int* iters, double* F, double* theta,
                  int* status, double* t_retire_ms)
{
    if (!b) return LGF_ERR_ARG;
    if (!(alpha > 0) || !(theta_tol >= 0) || max_iter < 0) return LGF_ERR_ARG;
    for (lgf_ctx* c : b->ctx)
        if (!c->have_links) return LGF_ERR_STATE;
    if (!b->tuned) {
        // tune each distinct lattice shape once (the choice is cached for the process)
        for (lgf_ctx* c : b->ctx) CKR(autotune_ctx(c));
        b->tuned = true;
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    CKR(batch_build(b));
    for (lgf_ctx* c : b->ctx) {
        *c->host_ctl = initial_ctl(c, alpha, theta_tol, max_iter);
        CK(cudaMemcpyAsync(c->ctl, c->host_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, b->stream));
    }
    CK(cudaGraphLaunch(b->exec, b->stream));
    for (lgf_ctx* c : b->ctx) CK(cudaMemcpyAsync(c->host_ctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(b->host_stamps.data(), b->stamps, b->host_stamps.size() * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaGetLastError());
    int worst = LGF_OK;
    for (size_t i = 0; i < b->ctx.size(); i++) {
        lgf_ctx* c = b->ctx[i];
        const Ctl r = *c->host_ctl;
        c->last_iters = r.iter;
        c->last_iters32 = r.iter_phase0;
        c->last_hist = r.iter + 1;
        const int st = status_of(r);
        if (iters) iters[i] = r.iter;
        if (F) F[i] = r.F;
        if (theta) theta[i] = r.theta;
        if (status) status[i] = st;
        if (t_retire_ms) t_retire_ms[i] = (double)(b->host_stamps[1 + i] - b->host_stamps[0]) * 1e-6;
        if (st != LGF_OK && worst == LGF_OK) worst = st;
    }
    return worst;
}

int lgf_batch_get_links(lgf_batch* b, int i, double* U_out, int on_device)
{
    if (!b || i < 0 || i >= (int)b->ctx.size()) return LGF_ERR_ARG;
    return lgf_get_links(b->ctx[i], U_out, on_device);
}

int lgf_batch_get_gauge(lgf_batch* b, int i, double* G_out, int on_device)
{
    if (!b || i < 0 || i >= (int)b->ctx.size()) return LGF_ERR_ARG;
    return lgf_get_gauge(b->ctx[i], G_out, on_device);
}

int lgf_batch_get_stats(lgf_batch* b, int i, int* iters_fp32, int* iters_fp64)
{
    if (!b || i < 0 || i >= (int)b->ctx.size()) return LGF_ERR_ARG;
    return lgf_get_stats(b->ctx[i], iters_fp32, iters_fp64);
}

int lgf_step_fwd(lgf_ctx* c, double alpha, const double* U_in, double* U_out)
{
    if (!c || !U_in || !U_out || !(alpha > 0)) return LGF_ERR_ARG;
    CKR(lgf_set_links(c, U_in, 1));
    int it = 0;
    const int r = lgf_fix(c, alpha, 0.0, 1, &it, nullptr, nullptr);
    // theta_tol = 0 is never met: one update and NOT_CONVERGED is the expected outcome
    if (r != LGF_ERR_NOT_CONVERGED && r != LGF_OK) return r;
    if (it != 1) return LGF_ERR_STATE;
    return lgf_get_links(c, U_out, 1);
}

int lgf_step_bwd(lgf_ctx* c, double alpha, const double* gU_out, double* gU_in)
{
    if (!c || !gU_out || !gU_in || !(alpha > 0)) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(ensure_diff(c));
    CKR(reset_stage_ctl(c, alpha));
    cudaStream_t s = c->stream;
    double2* Fd = reinterpret_cast<double2*>(c->Fd);
    // forward of the step on the stored links, up to g and the spatial Delta~
    launch_ah_init<double>(c->lat, s, c->U64, c->AH64, c->Fs64);
    launch_delta<double>(c->lat, c->sh64, c->tb, s, c->AH64, c->Fs64, Fd, c->partials, c->ctl_stage, nullptr, true);
    launch_zt<double>(c->lat, c->sh64, c->tb, s, Fd, c->ctl_stage);
    launch_xy_fft<double>(c->lat, c->sh64, c->tb, s, Fd, true);
    launch_g_from_dt(s, c->V, Fd, c->g64, alpha);
    // backward
    launch_pack_full(s, c->V, gU_out, c->dGp);
    launch_step_bwd(s, c->lat, c->U64, c->g64, Fd, c->dGp, c->dGud, c->dGgs, c->dQ, alpha, c->dFA, c->dFB);
    for (double2* F : {c->dFA, c->dFB}) {
        launch_xy_fft<double>(c->lat, c->sh64, c->tb, s, F, false);
        launch_zt<double>(c->lat, c->sh64, c->tb, s, F, c->ctl_stage);
        launch_xy_fft<double>(c->lat, c->sh64, c->tb, s, F, true);
    }
    launch_bwd_delta(s, c->lat, c->U64, c->dFA, c->dFB, c->dGud, c->dGp);
    launch_unpack_planes(s, c->V, c->dGp, gU_in);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return LGF_OK;
}

int lgf_gluon_pmin(lgf_ctx* c, double* D, double* Dp)
{
    if (!c || !D) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(ensure_gluon(c));
    launch_gluon(c->stream, c->lat, c->U64, c->tb, c->gl_part, c->gl_At, c->gl_D);
    double h[5];
    CK(cudaMemcpyAsync(h, c->gl_D, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    *D = h[4];
    if (Dp)
        for (int i = 0; i < 4; i++) Dp[i] = h[i];
    return LGF_OK;
}

int lgf_gluon_pmin_bwd(lgf_ctx* c, double gD, double* gU)
{
    if (!c || !gU) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(ensure_gluon(c));
    CKR(ensure_diff(c));
    // the forward's Fourier sums, then dD/dU
    launch_gluon(c->stream, c->lat, c->U64, c->tb, c->gl_part, c->gl_At, c->gl_D);
    const double coef = gD * 2.0 / (8.0 * 3.0 * (double)c->V) / 4.0 * 2.0;
    launch_gluon_bwd(c->stream, c->lat, c->U64, c->gl_At, coef, c->tb, c->dGp);
    launch_unpack_planes(c->stream, c->V, c->dGp, gU);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return LGF_OK;
}

int lgf_set_unit_links(lgf_ctx* c)
{
    if (!c) return LGF_ERR_ARG;
    if (c->lat.ne == 4) return LGF_ERR_STATE;  // the 8-real form cannot hold the unit matrix
    launch_unit_links(c->stream, c->lat, c->U64);
    if (c->track) launch_identity_rows64(c->stream, c->V, c->G64);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    c->have_links = true;
    return LGF_OK;
}

int lgf_wilson_sweeps(lgf_ctx* c, double beta, unsigned long long seed, int first_sweep, int n_heatbath,
                      int n_overrelax)
{
    if (!c || !(beta >= 0) || !std::isfinite(beta) || first_sweep < 0 || n_heatbath < 0 || n_overrelax < 0)
        return LGF_ERR_ARG;
    if (!c->have_links || c->lat.ne == 4) return LGF_ERR_STATE;  // the generator keeps 12 or 18 reals
    for (int mu = 0; mu < 4; mu++)
        if (c->L[mu] % 2) return LGF_ERR_UNSUPPORTED_DIMS;  // the checkerboard needs even extents
    if ((long long)first_sweep + n_heatbath > 0xffffffffLL) return LGF_ERR_ARG;
    if (c->gen_precision == 32) {
        if (!c->gen32) CKR(alloc((void**)&c->gen32, (size_t)24 * c->V * sizeof(float2)));
        launch_links_to_fp32(c->stream, c->lat, c->U64, c->gen32);
    }
    // n_heatbath = 0: overrelaxation sweeps only
    const int rounds = n_heatbath > 0 ? n_heatbath : 1;
    for (int i = 0; i < rounds; i++) {
        const unsigned int sweep = (unsigned int)(first_sweep + i);
        for (int mode = n_heatbath > 0 ? 0 : 1; mode < 1 + n_overrelax; mode++)
            for (int mu = 0; mu < 4; mu++)
                for (int par = 0; par < 2; par++)
                    launch_wilson(c->stream, c->lat, c->U64, c->gen32, mu, par, mode > 0, beta, seed, sweep,
                                  c->gen_precision);
        CK(cudaGetLastError());
    }
    if (c->track) launch_identity_rows64(c->stream, c->V, c->G64);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return LGF_OK;
}

int lgf_set_generator_precision(lgf_ctx* c, int bits)
{
    if (!c || (bits != 64 && bits != 32)) return LGF_ERR_ARG;
    c->gen_precision = bits;
    return LGF_OK;
}

int lgf_plaquette(lgf_ctx* c, double* P)
{
    if (!c || !P) return LGF_ERR_ARG;
    if (!c->have_links) return LGF_ERR_STATE;
    CKR(ensure_plaq(c));
    const int nb = plaquette_blocks(c->V);
    launch_plaquette(c->stream, c->lat, c->U64, c->wil_part, c->wil_part + nb);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(P, c->wil_part + nb, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LGF_OK;
}

}  // extern "C"
