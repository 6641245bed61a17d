// Allocation-free variant of the FP64 primal-residual yardstick (ddh_primal_residual).
//
// Some callers cannot allocate device memory at the point where they need this number.
// An application that reserves its whole device-memory budget at start-up (its own pool
// allocator, or a hard cap shared with other solvers on the same GPU) forbids any later
// cudaMalloc: the allocation would fail or break its accounting.  A caller inside a
// latency-critical loop avoids cudaMalloc and cudaFree because they can synchronise the
// whole device and stall the work of other streams.  This entry point works in one
// file-scope scratch array in device memory instead of the context's on-demand work
// buffers, so it allocates nothing.  The array is a symbol of this library: every GPU
// that loads the library holds kScratchBytes of it until the process exits.  The call
// still synchronises the context stream to return the norms to the host, so it refuses to
// run while that stream is being captured into a CUDA graph.
#include <mutex>

#include "../../include/ddh.h"
#include "ddh_launch.hpp"

namespace ddh {
// context accessors (defined next to the context in ddh_api.cu)
const DevModel* ctx_devmodel(ddh_ctx* c);
cudaStream_t ctx_stream(ddh_ctx* c);
int ctx_device(ddh_ctx* c);
bool ctx_factored(ddh_ctx* c);
void ctx_set_error(ddh_ctx* c, const char* msg);
void ctx_add_launches(ddh_ctx* c, int n);
}  // namespace ddh

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxRhs = 512;

// Scratch shared by every call on a device.  In host code `g_scratch` only names the symbol
// (a host-side stand-in, not a device address): kernels get the address returned by
// cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Makes `dev` current for the lifetime of the guard and gives the caller's current device
// back on every return path.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" ddh_status ddh_primal_residual_noalloc(ddh_ctx* ctx, const void* b_dev, const void* u_dev, int32_t R,
                                                  double* out_host) {
    using namespace ddh;
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx_factored(ctx)) { ctx_set_error(ctx, "factor first"); return DDH_ERR_NOT_READY; }
    if (!b_dev || !u_dev || !out_host || R <= 0) { ctx_set_error(ctx, "bad arguments"); return DDH_ERR_INVALID_ARG; }
    if (R > kMaxRhs) { ctx_set_error(ctx, "ddh_primal_residual_noalloc: at most 512 right-hand sides"); return DDH_ERR_INVALID_ARG; }
    const DevModel& d = *ctx_devmodel(ctx);
    const int dev = ctx_device(ctx);
    if (dev < 0 || dev >= kMaxDevices) { ctx_set_error(ctx, "device index out of range"); return DDH_ERR_INVALID_ARG; }
    // scratch layout: b~, phi~, u_c, phi_c, r (local/conforming vectors), two norm accumulators
    const size_t loc = align256(sizeof(double2) * (size_t)R * d.n_local);
    const size_t conf = align256(sizeof(double2) * (size_t)R * d.n_conf);
    const size_t nrm = align256(sizeof(double) * (size_t)R);
    const size_t need = 4 * loc + conf + 2 * nrm;
    if (need > kScratchBytes) {
        ctx_set_error(ctx, "ddh_primal_residual_noalloc: this mesh and R need more than the 32 MiB allocation-free "
                           "scratch (4 R n_local + R n_conforming complex128); use ddh_primal_residual");
        return DDH_ERR_INVALID_ARG;
    }
    const DeviceGuard guard(dev);
    if (!guard.ok) { ctx_set_error(ctx, "cudaSetDevice failed"); return DDH_ERR_CUDA; }
    {
        // the call ends with a host read of the norms (a stream synchronisation), which a stream
        // capture cannot hold: refuse before touching the stream, and leave the capture intact
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(ctx_stream(ctx), &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            ctx_set_error(ctx, "ddh_primal_residual_noalloc: the context stream is being captured; the call "
                               "synchronises the stream and cannot be captured");
            return DDH_ERR_INVALID_ARG;
        }
    }
    unsigned char* base;
    {
        // once per device, with that device current: the device address of the scratch symbol
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                ctx_set_error(ctx, cudaGetErrorString(e));
                return DDH_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        base = (unsigned char*)g_scratch_addr[dev];
    }
    double2* bt = (double2*)base;
    double2* pt = (double2*)(base + loc);
    double2* phc = (double2*)(base + 2 * loc);
    double2* res = (double2*)(base + 3 * loc);
    double2* uc = (double2*)(base + 4 * loc);
    double* n1 = (double*)(base + 4 * loc + conf);
    double* n2 = (double*)(base + 4 * loc + conf + nrm);
    cudaStream_t s = ctx_stream(ctx);
    // the array keeps the previous call's contents: clear the accumulators
    if (cudaMemsetAsync(n1, 0, 2 * nrm, s) != cudaSuccess) { ctx_set_error(ctx, "cudaMemsetAsync failed"); return DDH_ERR_CUDA; }
    launch_basis(d, (const double2*)b_dev, bt, 0, R, s);
    launch_basis(d, (const double2*)u_dev, pt, 0, R, s);
    launch_readback(d, pt, uc, R, s);
    launch_conf_scatter(d, uc, phc, R, s);
    launch_elem_matvec(d, phc, bt, res, R, s);
    launch_conf_gather(d, res, n1, R, s);
    launch_conf_gather(d, bt, n2, R, s);
    ctx_add_launches(ctx, 7);
    double a[kMaxRhs], b[kMaxRhs];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(a, n1, sizeof(double) * R, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b, n2, sizeof(double) * R, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { ctx_set_error(ctx, cudaGetErrorString(e)); return DDH_ERR_CUDA; }
    for (int i = 0; i < R; ++i) out_host[i] = b[i] > 0 ? sqrt(a[i] / b[i]) : sqrt(a[i]);
    return DDH_OK;
}
