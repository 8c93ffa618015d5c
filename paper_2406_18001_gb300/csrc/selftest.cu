// selftest.cu -- failure-path hooks of libdcd_gb300.so, for testing how the
// library reports failures without faulting, trapping or hanging a GPU.
//
// dcd_selftest_bounded_wait: every wait on an mbarrier in the library's
// kernels is bounded; when the bound runs out the kernel records DEV_TIMEOUT
// in the device error word, stops waiting and returns, and the host turns the
// word into DCD_ETIMEOUT.  The self-test runs that path for real: one thread
// waits, with the library's bounded wait, on an mbarrier whose arrival count
// (2) is never reached (one arrival).
//
// dcd_inject_alloc_failures: the next `count` device allocations the library
// makes fail as if the device were out of memory (DCD_ENOMEM), a fake of the
// failing call made on the host.
#include "dcd_internal.cuh"
#include "ptx.cuh"

#include <atomic>

namespace dcd {
namespace {

std::atomic<int> g_fail_allocs{0};

__global__ void bounded_wait_selftest_kernel(unsigned long long limit_ns, int *err, int *waited)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    ptx::mbar_init(&bar, 2);
    ptx::mbar_init_fence();
    ptx::mbar_arrive(&bar);  // one of the two arrivals the phase needs
    const bool done = ptx::mbar_wait_bounded(&bar, 0, limit_ns);
    *waited = 1;
    if (!done) set_error(err, DEV_TIMEOUT);
}

}  // namespace

cudaError_t malloc_async(void **p, size_t bytes, cudaStream_t st)
{
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMallocAsync(p, bytes, st);
}

}  // namespace dcd

using namespace dcd;

extern "C" dcd_status dcd_inject_alloc_failures(int32_t count)
{
    if (count < 0) return DCD_EINVAL;
    g_fail_allocs.store(count);
    return DCD_OK;
}

extern "C" dcd_status dcd_selftest_bounded_wait(int64_t limit_ns, void *stream)
{
    if (limit_ns < 1000 || limit_ns > 1000000000) return DCD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int *d = nullptr;
    cudaError_t e = malloc_async((void **)&d, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DCD_ENOMEM : DCD_ECUDA;
    int h[2] = {0, 0};
    e = cudaMemsetAsync(d, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        bounded_wait_selftest_kernel<<<1, 32, 0, st>>>((unsigned long long)limit_ns, d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DCD_ECUDA;
    if (!h[1]) return DCD_EINTERNAL;  // the kernel did not reach its wait
    return h[0] == DEV_TIMEOUT ? DCD_ETIMEOUT : h[0] ? DCD_EINTERNAL : DCD_OK;
}
