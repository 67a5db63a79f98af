// noalloc.cu - ssm_gram_pair without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns every byte of device memory through its own pool, code on
// a latency-critical path where cudaMalloc's implicit device
// synchronisation is not acceptable, or plug-ins whose host forbids raw
// CUDA allocations.  For them this file keeps the partial sums of the Gram
// pair in a fixed, file-scope device array instead of a cudaMalloc'd buffer.
//
// The array is 4 MiB of float64 (524288 values).  Every GPU that loads the
// library holds it until the process exits.  A call needs
// 2 * n_cols^2 values per row slice and uses as many slices as fit (at most
// the number ssm_gram_pair would use), so n_cols is limited to 512.
#include <mutex>

#include "internal.h"

namespace ssm {

namespace {

constexpr size_t NOALLOC_PART_VALUES = 524288;  // 4 MiB of double
constexpr int NOALLOC_MAX_COLS = 512;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Shared by every call on a device; holds the last call's partial sums.
static __device__ __align__(256) double g_noalloc_part[NOALLOC_PART_VALUES];

// Device address of g_noalloc_part per device (the host-side name of the array
// is only a stand-in and must never be passed to a kernel).  A device's primary
// context can be destroyed and made again (cudaDeviceReset), which loads the
// module anew at another address, so outside stream capture the address is
// looked up on every call (cudaGetSymbolAddress allocates nothing); while the
// stream is being captured the last looked-up address is used.
void* g_part_addr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_part_mutex;

cudaError_t part_address(int device, cudaStream_t stream, double** out) {
    std::lock_guard<std::mutex> lock(g_part_mutex);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs == cudaStreamCaptureStatusNone || !g_part_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess) return e;
        g_part_addr[device] = p;
    }
    *out = (double*)g_part_addr[device];
    return cudaSuccess;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace ssm

extern "C" ssm_status ssm_gram_pair_noalloc(const double* A, const double* B, int64_t n_rows, int32_t n_cols,
                                            int64_t ld, double* G_aa, double* G_ab, void* stream) {
    using namespace ssm;
    auto reject = [](ssm_status st, const char* msg) {
        set_global_error(msg);
        return st;
    };
    if (!A || !G_aa || (B && !G_ab)) return reject(SSM_EINVAL, "A and G_aa (and G_ab with B) are required");
    if (n_rows < 0 || n_cols < 1 || ld < n_cols || ld > INT32_MAX)
        return reject(SSM_EINVAL, "need n_rows >= 0, n_cols >= 1, n_cols <= ld < 2^31");
    if (n_cols > NOALLOC_MAX_COLS)
        return reject(SSM_EINVAL, "ssm_gram_pair_noalloc: n_cols exceeds 512, the size its fixed 4 MiB scratch holds");
    if (!on_device(A) || (B && !on_device(B)) || !on_device(G_aa) || (G_ab && !on_device(G_ab)))
        return reject(SSM_EINVAL, "ssm_gram_pair_noalloc takes device pointers only");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= NOALLOC_MAX_DEVICES)
        return reject(SSM_ECUDA, "no usable current device");
    double* part = nullptr;
    if (part_address(device, (cudaStream_t)stream, &part) != cudaSuccess)
        return reject(SSM_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed");
    const size_t per_split = (size_t)2 * n_cols * n_cols;
    int n_split = gram_split_count(n_rows, n_cols);
    const int fit = (int)(NOALLOC_PART_VALUES / per_split);
    if (n_split > fit) n_split = fit;
    cudaStream_t s = (cudaStream_t)stream;
    if (launch_gram_f64(A, B, (int)ld, n_cols, n_rows, n_split, part, s) != cudaSuccess)
        return reject(SSM_ECUDA, "Gram kernel launch failed");
    if (launch_reduce_gram_pair(part, n_split, n_cols, G_aa, B ? G_ab : nullptr, s) != cudaSuccess)
        return reject(SSM_ECUDA, "reduction kernel launch failed");
    return SSM_OK;
}
