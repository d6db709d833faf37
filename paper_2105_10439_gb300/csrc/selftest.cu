// Self-test of the bounded on-device waits.  The persistent kernels wait on
// other CTAs (a grid-wide counter in the single-pass operator) and on their
// own pipeline (mbarriers of the tensor-core GEMMs); every such wait gives up
// after a limit, sets COFEM_FLAG_DEVICE_TIMEOUT and lets the kernel return, so
// that a fit reports COFEM_ERR_CUDA instead of hanging the GPU.  This kernel
// runs the same two wait routines (tc_ptx.cuh) on a counter and an mbarrier
// that nothing completes, with short limits, so the reporting path can be
// checked on a GPU without a fault or a hang: both waits end by their limits.
#include "cofem_internal.cuh"
#include "tc_ptx.cuh"

namespace {

__global__ void k_wait_selftest(const unsigned* ctr, unsigned* flags, unsigned long long grid_ns,
                                unsigned mbar_rounds, int* result) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(smem_u32(&bar), 1);   // one arrival completes phase 0; none comes
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const bool g = grid_wait(ctr, 1u, &abort_flag, flags, grid_ns);   // nothing raises *ctr
    abort_flag = 0;
    const bool m = mbar_wait(smem_u32(&bar), 0u, &abort_flag, mbar_rounds);
    if (!g || !m) atomicOr(flags, COFEM_FLAG_DEVICE_TIMEOUT);
    result[0] = g ? 1 : 0;
    result[1] = m ? 1 : 0;
}

}  // namespace

extern "C" cofem_status cofem_selftest_bounded_wait(double seconds, unsigned* flags_out) {
    if (!(seconds >= 1e-3 && seconds <= 2.0))
        return cofem_set_error(COFEM_ERR_INVALID_ARG, "need 1e-3 <= seconds <= 2");
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 16);
    if (e != cudaSuccess) return cofem_set_error(COFEM_ERR_NOMEM, cudaGetErrorString(e));
    unsigned* ctr = (unsigned*)buf;
    unsigned* flags = ctr + 1;
    int* result = (int*)(ctr + 2);
    int host[2] = {-1, -1};
    unsigned hflags = 0;
    if ((e = cudaMemset(buf, 0, 16)) == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(ctr, flags, (unsigned long long)(seconds * 1e9), 4096u, result);
        if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaDeviceSynchronize()) == cudaSuccess &&
            (e = cudaMemcpy(host, result, sizeof(host), cudaMemcpyDeviceToHost)) == cudaSuccess)
            e = cudaMemcpy(&hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost);
    }
    cudaFree(buf);
    if (e != cudaSuccess) return cofem_set_error(COFEM_ERR_CUDA, cudaGetErrorString(e));
    if (flags_out) *flags_out = hflags;
    if (hflags & COFEM_FLAG_DEVICE_TIMEOUT)
        return cofem_set_error(COFEM_ERR_CUDA,
                               host[0] == 0 && host[1] == 0
                                   ? "a bounded on-device wait timed out (grid counter and mbarrier self-test)"
                                   : "a bounded on-device wait timed out (self-test)");
    return COFEM_OK;
}
