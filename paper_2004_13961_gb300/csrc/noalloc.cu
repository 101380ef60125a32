// noalloc.cu -- lsg_gauss_noalloc: the Legendre-Gauss rule without any device
// allocation.
//
// lsg_gauss allocates two device buffers on every call for the kernel to write
// the nodes and weights into before they are copied to the caller's host
// arrays.  Some callers cannot allocate device memory at call time: code that
// runs while the device's memory is fully reserved by another component, or
// under a policy that forbids allocator calls once a job has started (for
// instance a latency-critical loop where an allocation could block on the
// driver).  For them this variant keeps that scratch in a file-scope device
// array of fixed size instead.
#include <mutex>
#include <stdio.h>

#include "lsg_internal.cuh"

namespace {

// Largest Q served: two arrays of Q doubles (256 KiB in total on every device
// that loads the library, held until the process exits).
constexpr int kNoAllocMaxQ = 16384;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gauss_scratch[2 * kNoAllocMaxQ];

std::mutex g_scratch_mu;
double *g_scratch_dev[kMaxDevices] = {};

}  // namespace

extern "C" int lsg_gauss_noalloc(int Q, double *x, double *w)
{
    if (Q < 1 || !x || !w) return LSG_ERR_ARG;
    if (Q > kNoAllocMaxQ) {
        cudaError_t e = cudaErrorInvalidValue;
        lsg::record_cuda_error(e, "lsg_gauss_noalloc: Q exceeds the static scratch limit of 16384 points",
                               __FILE__, __LINE__);
        return LSG_ERR_ARG;
    }
    int dev = 0;
    LSG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        lsg::record_cuda_error(cudaErrorInvalidDevice, "lsg_gauss_noalloc: device index beyond the 64 devices it keeps a scratch address for",
                               __FILE__, __LINE__);
        return LSG_ERR_ARG;
    }
    double *base = nullptr;
    {
        // once per device, with that device current: the host-side symbol is only a
        // stand-in, so look up the array's device address before any kernel gets it
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_gauss_scratch);
            if (e != cudaSuccess) {
                lsg::record_cuda_error(e, "cudaGetSymbolAddress(g_gauss_scratch)", __FILE__, __LINE__);
                return LSG_ERR_CUDA;
            }
            g_scratch_dev[dev] = (double *)p;
        }
        base = g_scratch_dev[dev];
    }
    // the kernel writes all Q nodes and weights, so nothing needs clearing first
    int st = lsg::gauss_rule(Q, base, base + kNoAllocMaxQ, 0);
    if (st != LSG_OK) return st;
    LSG_CK(cudaMemcpy(x, base, sizeof(double) * Q, cudaMemcpyDeviceToHost));
    LSG_CK(cudaMemcpy(w, base + kNoAllocMaxQ, sizeof(double) * Q, cudaMemcpyDeviceToHost));
    return LSG_OK;
}
