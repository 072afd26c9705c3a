// Self-test of the bounded device-side wait that every staged kernel of the library uses
// (see az_selftest_wait in azint.h): a one-warp kernel waits on a shared-memory barrier that
// nothing completes (or that its first thread completes, as a control) and reports, instead
// of hanging, that the wait gave up.
#include "common.cuh"

using namespace azint;

namespace {

constexpr long long kSelftestMaxCycles = 2000000000LL;  // about one second of the SM clock

__global__ void wait_selftest_kernel(int arrive, long long limit, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar, 0u, limit));
    if (threadIdx.x == 0) *status = ok ? AZ_OK : AZ_ETIMEOUT;
}

}  // namespace

extern "C" int az_selftest_wait(int arrive, int64_t limit_cycles, int *out_status, az_stream_t stream) {
    clear_error();
    if (!out_status) return fail(AZ_EINVAL, "az_selftest_wait: NULL status");
    if (limit_cycles <= 0 || limit_cycles > kSelftestMaxCycles)
        return fail(AZ_EINVAL, "az_selftest_wait: limit_cycles must be in (0, %lld]", kSelftestMaxCycles);
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf st;
    AZ_TRY(st.alloc(sizeof(int)));
    AZ_CUDA(cudaMemsetAsync(st.p, 0xff, sizeof(int), s));  // -1 until the kernel writes
    wait_selftest_kernel<<<1, 32, 0, s>>>(arrive ? 1 : 0, (long long)limit_cycles, st.as<int>());
    AZ_CUDA(cudaGetLastError());
    int v = 0;
    AZ_CUDA(cudaMemcpyAsync(&v, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    *out_status = v;
    return AZ_OK;
}
