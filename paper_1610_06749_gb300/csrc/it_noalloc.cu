// it_noalloc.cu -- one explicit step that allocates no device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or a plugin that is only handed buffers, and
// long-running services that must not allocate once they are up (an
// allocation can fail, fragment the pool, or synchronise the device at a
// bad moment).  it_step_noalloc serves them: the caller passes the input
// and output densities and the tally output; the per-block tally partials
// the step kernel needs live in a fixed array in this file's device
// memory, so nothing is allocated.
//
// The array: IT_NOALLOC_MAX_BLOCKS x 10 doubles (160 KiB), held by every
// GPU that loads the library until the process exits.  Its device address
// is looked up once per device (cudaGetSymbolAddress, with that device
// current) on the first call made on that device; that first call should
// therefore come before any stream capture.  Every call shares the array
// and zeroes the part it uses before the step, so two calls that overlap on
// the GPU (different streams, or different host threads, without ordering
// between them) race on it and must not be issued.
#include <mutex>

#include "it_device.cuh"
#include "it_internal.cuh"

namespace itk {

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_slots[IT_NOALLOC_MAX_BLOCKS * NT];

std::mutex g_noalloc_mu;
double *g_noalloc_addr[kMaxDevices];

// device address of g_noalloc_slots on the current device (looked up once)
int noalloc_scratch(double **out) {
    int dev = 0;
    IT_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("it_step_noalloc: device index beyond the supported 64 devices");
        return IT_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_slots);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc tally scratch)");
        g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[dev];
    return IT_OK;
}

// Fixed-order sum of the per-block slots into the 7 tallies of this step
// (same order as the context's finalize reduction).
__global__ void __launch_bounds__(256)
noalloc_reduce_kernel(const double *__restrict__ slots, int nslots, double *__restrict__ out7) {
    __shared__ double red[32 * 7];
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nslots; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 7; ++q) v[q] += slots[(size_t)b * NT + q];
    }
    block_sum<7>(v, red);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 7; ++q) out7[q] = v[q];
    }
}

}  // namespace

}  // namespace itk

using namespace itk;

extern "C" int it_step_noalloc(it_grid g, double dx_cm, double dt_s, const it_params *p, const float *dev_plus,
                               const float *dev_minus, float *dev_out_plus, float *dev_out_minus,
                               double *dev_tallies7, void *stream) {
    int rc = validate_step_args(p, g, dx_cm, dt_s);
    if (rc) return rc;
    if (p->precision != IT_FP32) {
        set_error("it_step_noalloc: FP32 densities only");
        return IT_EINVAL;
    }
    if (p->space_charge) {
        set_error("it_step_noalloc: the space-charge term is not available here (its tallies are not among the 7)");
        return IT_EINVAL;
    }
    if (!dev_plus || !dev_minus || !dev_out_plus || !dev_out_minus || !dev_tallies7) {
        set_error("it_step_noalloc: NULL buffer");
        return IT_EINVAL;
    }
    if (dev_plus == dev_out_plus || dev_minus == dev_out_minus || dev_plus == dev_out_minus ||
        dev_minus == dev_out_plus) {
        set_error("it_step_noalloc: outputs must not alias the inputs");
        return IT_EINVAL;
    }
    const size_t cells = (size_t)g.nx * g.ny * g.nz;
    int dev = 0, sms = 0;
    IT_CK(cudaGetDevice(&dev));
    IT_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t want = (cells + 255) / 256;
    const size_t cap = (size_t)sms * 8;
    const size_t blocks = want < cap ? want : cap;
    if (blocks > (size_t)IT_NOALLOC_MAX_BLOCKS) {
        set_error("it_step_noalloc: this device needs " + std::to_string(blocks) +
                  " tally blocks, the static scratch holds " + std::to_string(IT_NOALLOC_MAX_BLOCKS));
        return IT_EINVAL;
    }
    double *slots = nullptr;
    rc = noalloc_scratch(&slots);
    if (rc) return rc;
    Coef<float> cf;
    coef_f32(p, dx_cm, dt_s, &cf);
    cudaStream_t s = (cudaStream_t)stream;
    // the step kernel adds into its slots: clear the part this call uses
    IT_CK(cudaMemsetAsync(slots, 0, sizeof(double) * NT * blocks, s));
    rc = launch_step_simple_raw_f32(dev_plus, dev_minus, dev_out_plus, dev_out_minus, g.nx, g.ny, g.nz, cf,
                                    p->lateral_bc == IT_PERIODIC, slots, (int)blocks, s);
    if (rc) return rc;
    noalloc_reduce_kernel<<<1, 256, 0, s>>>(slots, (int)blocks, dev_tallies7);
    IT_CK(cudaGetLastError());
    return IT_OK;
}
