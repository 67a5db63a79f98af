// selftest.cu - the bounded mbarrier wait of the tensor-core kernels, on its own.
//
// Every spin or suspend on an mbarrier in this library stops after a bounded
// number of polls and reports the failure in a status word instead of hanging
// the GPU.  This kernel runs that mechanism with nothing else in flight (no
// bulk copy, no MMA): one thread initialises an mbarrier expecting one
// arrival, optionally arrives, then waits for the phase with at most `polls`
// tests.  Without the arrival the wait must give up, and the kernel returns
// normally with *status = 1.
#include "internal.h"
#include "tcgen05.cuh"

namespace ssm {

namespace {

__global__ void selftest_wait_kernel(int polls, int arrive, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (arrive) tc::mbar_arrive(&bar);
    bool done = false;
    for (int i = 0; i < polls && !done; ++i) done = tc::mbar_test(tc::smem_u32(&bar), 0);
    *status = done ? 0 : 1;
}

}  // namespace

cudaError_t launch_selftest_wait(int polls, bool arrive, int* status, cudaStream_t s) {
    selftest_wait_kernel<<<1, 32, 0, s>>>(polls, arrive ? 1 : 0, status);
    return cudaGetLastError();
}

}  // namespace ssm
