// ap_grad_quadforms_static: the MLL-gradient quadratic forms of
// ap_grad_quadforms without any device allocation.
//
// Why it exists: ap_grad_quadforms may grow context work buffers with
// cudaMalloc on its first use with a given size.  Some callers cannot let that
// happen once their steady state has begun: latency-bound serving loops
// (cudaMalloc and cudaFree synchronise the whole device, stalling every other
// stream) and processes whose own memory pool already holds all free HBM (a
// cudaMalloc would fail).  They build the context once at set-up and then call
// this entry point, which uses only the buffers the caller passes and one
// fixed scratch array compiled into the library.  The call still copies its
// sums to the host and synchronises the context's stream before returning.
#include <mutex>

#include "ap_internal.cuh"

namespace ap {
namespace {

// Fixed scratch of the gradient kernel: per-CTA partial sums, the finishing
// ticket and the final sums.  Every GPU that loads libap.so holds it until the
// process exits.  Zero-initialised at module load; the ticket is cleared again
// before every launch, the partials and sums are fully rewritten by each call.
constexpr size_t kScratchDoubles = (size_t)AP_STATIC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr size_t kTicketOff = 0;   // one unsigned int (padded to 8 doubles)
constexpr size_t kOutOff = 8;      // D + 2 <= 34 sums
constexpr size_t kPartOff = 64;    // per-CTA partials

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

// Device address of g_scratch on device `dev`, which must be current; looked
// up once per device (a host-side name of a __device__ array is not a device
// address).
cudaError_t scratch_on_device(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
        if (err != cudaSuccess) return err;
        g_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace ap

using namespace ap;

extern "C" ap_status ap_grad_quadforms_static(ap_ctx* ctx, const float* U_dev, const float* V_dev, int32_t c,
                                              const double* alpha_host, double* out_host) {
    if (!ctx || !U_dev || !V_dev || !alpha_host || !out_host) return AP_ERR_INVALID_ARG;
    if (c != 1 && c != 4 && c != 16 && c != 32) return AP_ERR_INVALID_ARG;
    GradView v;
    ctx_grad_view(ctx, &v);
    const int NA = v.D + 2;
    const int64_t rows = grad_rows_per_cta(v.D, c);
    const int64_t ntiles = (v.n + rows - 1) / rows;
    if ((size_t)(kPartOff + ntiles * NA) > kScratchDoubles) return AP_ERR_SCRATCH_LIMIT;
    DeviceGuard dg(v.device);  // the context's device is current for the look-up and the launch
    if (!dg.ok()) return AP_ERR_CUDA;
    double* scratch = nullptr;
    if (scratch_on_device(v.device, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return AP_ERR_CUDA;
    }
    GradParams gp = {};
    gp.Xs = v.Xs;
    gp.n = v.n;
    gp.U = U_dev;
    gp.V = V_dev;
    for (int k = 0; k < c; ++k) gp.alpha[k] = (float)alpha_host[k];
    gp.ntiles = ntiles;
    gp.S = 1;
    gp.part = scratch + kPartOff;
    gp.ticket = reinterpret_cast<unsigned int*>(scratch + kTicketOff);
    gp.out = scratch + kOutOff;
    double raw[AP_MAX_DIM + 2] = {};
    if (cudaMemsetAsync(gp.ticket, 0, sizeof(unsigned int), v.stream) != cudaSuccess ||
        launch_grad(v.kernel, gp, v.D, c, v.stream) != cudaSuccess ||
        cudaMemcpyAsync(raw, gp.out, sizeof(double) * NA, cudaMemcpyDeviceToHost, v.stream) != cudaSuccess ||
        cudaStreamSynchronize(v.stream) != cudaSuccess) {
        cudaGetLastError();
        return AP_ERR_CUDA;
    }
    grad_finish(v, raw, out_host);
    return AP_OK;
}
