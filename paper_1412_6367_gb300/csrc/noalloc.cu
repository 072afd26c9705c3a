// Single-frame forward whose scratch lives in a fixed array compiled into this library, for
// callers that must not allocate device memory while they run (see az_integrate_noalloc in
// azint.h).  The kernels are the ones az_integrate1d / az_integrate2d launch; only the
// buffer that holds the per-segment partial sums between the two phases differs.
#include <mutex>

#include "common.cuh"

using namespace azint;

namespace {

// The partial sums of one call: 3 quantities (signal, normalisation, count) per segment.
// Every GPU that loads this library reserves this much memory for it until the process exits.
static __device__ __align__(256) unsigned char g_partial_scratch[AZ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];  // device address of g_partial_scratch, per device

// Host code may not hand the array's name to a kernel: on the host that name is a stand-in,
// not the device address.  Look the address up once per device, with that device current.
int scratch_address(void **out) {
    int dev = 0;
    AZ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(AZ_EUNSUPPORTED, "az_integrate_noalloc: device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partial_scratch);
        if (e != cudaSuccess || !p)
            return fail(AZ_ECUDA, "az_integrate_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return AZ_OK;
}

bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

}  // namespace

namespace azint {
// Set-up on the current device, run when an integrator is built there: the array's address
// is looked up (under the CUDA runtime's lazy module loading this is what loads this file's
// module and reserves the array) and the kernels of the single-pass forward are loaded, so
// that the entry point's calls themselves take no device memory.
int noalloc_setup() {
    void *p = nullptr;
    AZ_TRY(scratch_address(&p));
    return preload_single_pass();
}
}  // namespace azint

extern "C" int az_integrate_noalloc(const az_integrator *h, const void *image_dev, int image_dtype,
                                    const float *dark, const float *flat, const float *solid_angle,
                                    const float *polarization, int precision, void *out_I,
                                    void *out_sum_signal, void *out_sum_norm, void *out_count,
                                    az_stream_t stream) {
    clear_error();
    const char *who = "az_integrate_noalloc";
    if (!h) return fail(AZ_EINVAL, "%s: NULL integrator", who);
    if (!image_dev) return fail(AZ_EINVAL, "%s: NULL image", who);
    if (image_dtype < AZ_DTYPE_F32 || image_dtype > AZ_DTYPE_I32)
        return fail(AZ_EINVAL, "%s: bad image dtype %d", who, image_dtype);
    const void *ptrs[5] = {image_dev, dark, flat, solid_angle, polarization};
    for (const void *p : ptrs)
        if (p && !aligned4(p)) return fail(AZ_EINVAL, "%s: arrays must be 4-byte aligned", who);
    if (precision != AZ_PREC_FP64 && precision != AZ_PREC_FP32_COMP)
        return fail(AZ_EINVAL, "%s: bad precision %d", who, precision);
    const size_t value_bytes = precision == AZ_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = 3 * (size_t)h->tl.nseg * value_bytes;
    if (need > (size_t)AZ_NOALLOC_SCRATCH_BYTES)
        return fail(AZ_ESHAPE,
                    "%s: this integrator needs %zu bytes of partial sums (%d segments x 3 x %zu bytes) "
                    "but the library's fixed buffer holds %zu; use az_integrate1d/2d, FP32, or larger tiles",
                    who, need, h->tl.nseg, value_bytes, (size_t)AZ_NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    AZ_TRY(scratch_address(&scratch));
    const_cast<az_integrator *>(h)->last_stream = (cudaStream_t)stream;
    return forward_single_into(h, image_dev, image_dtype, dark, flat, solid_angle, polarization,
                               precision, out_I, out_sum_signal, out_sum_norm, out_count, scratch,
                               (cudaStream_t)stream);
}
