// Allocation-free variant of the dense operator application
// Psi = beta Phi^T (Phi V) + diag(alpha) V, for callers that cannot allocate
// device memory.  The intermediate T = Phi V (N x Q floats) lives in a
// file-scope __device__ array of fixed size instead of a cudaMalloc'd buffer;
// every caller on a device shares that array.
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "cofem_internal.cuh"

namespace {

// Scratch for T = Phi V, row-major N x Q.  Every device that loads the library
// holds these COFEM_NOALLOC_MAX_ELEMS floats (4 MiB) until the process exits.
__device__ __align__(256) float g_noalloc_T[COFEM_NOALLOC_MAX_ELEMS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
// Per device: the scratch address and the CUDA context it was looked up in.
// A device reset (cudaDeviceReset) ends that context and may move the array,
// so the address is looked up again when the current context differs.
float* g_na_scratch[NA_MAX_DEVICES] = {};
CUcontext g_na_ctx[NA_MAX_DEVICES] = {};

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);

// The current CUDA context of this thread (the runtime makes the device's
// primary context current on its first call), through the driver entry point
// the runtime hands out, so the library needs no link to libcuda.
cofem_status na_current_context(CUcontext* out) {
    static PfnCtxGetCurrent fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f)
            return cofem_set_error(COFEM_ERR_CUDA, "cuCtxGetCurrent is not available from the CUDA driver");
        fn = (PfnCtxGetCurrent)f;
    }
    if (fn(out) != CUDA_SUCCESS) return cofem_set_error(COFEM_ERR_CUDA, "cuCtxGetCurrent failed");
    return COFEM_OK;
}

// Device address of the scratch array on the current device.  The array's name
// in host code is only a host-side stand-in, so the address is looked up with
// that device current: once per device and context.
cofem_status na_scratch(int dev, float** out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cofem_set_error(COFEM_ERR_UNSUPPORTED, "device index too large");
    // the runtime calls before this one (cudaGetDevice, cudaPointerGetAttributes)
    // have made the device's primary context current on this thread
    CUcontext ctx = nullptr;
    cofem_status st = na_current_context(&ctx);
    if (st) return st;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_scratch[dev] || g_na_ctx[dev] != ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_T);
        if (e != cudaSuccess) {
            char msg[160];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            return cofem_set_error(COFEM_ERR_CUDA, msg);
        }
        g_na_scratch[dev] = (float*)p;
        g_na_ctx[dev] = ctx;
    }
    *out = g_na_scratch[dev];
    return COFEM_OK;
}

// Device (or managed) memory that the current device `dev` can address: device
// memory of another GPU is refused (it would fault without peer access).
bool is_device_memory(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

constexpr int NA_QB = 8;     // columns per pass of the first kernel
constexpr int NA_QB2 = 16;   // columns per block of the second kernel

// T[i][q] = sum_j Phi[i][j] V[q][j]: one block per row i, NA_QB columns per pass.
__global__ __launch_bounds__(256) void k_na_phiv(const float* __restrict__ phi, long long N, long long D,
                                                 long long ld, const float* __restrict__ V, int Q,
                                                 float* __restrict__ T) {
    __shared__ float red[NA_QB][8];
    const long long i = blockIdx.x;
    const float* row = phi + i * ld;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q0 = 0; q0 < Q; q0 += NA_QB) {
        float acc[NA_QB];
#pragma unroll
        for (int k = 0; k < NA_QB; ++k) acc[k] = 0.0f;
        for (long long j = threadIdx.x; j < D; j += blockDim.x) {
            const float a = row[j];
#pragma unroll
            for (int k = 0; k < NA_QB; ++k)
                if (q0 + k < Q) acc[k] = fmaf(a, V[(size_t)(q0 + k) * D + j], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < NA_QB; ++k) {
            float v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[k][w] = v;
        }
        __syncthreads();
        if (threadIdx.x < NA_QB && q0 + threadIdx.x < Q) {
            float v = 0.0f;
            for (int ww = 0; ww < 8; ++ww) v += red[threadIdx.x][ww];
            T[i * Q + q0 + threadIdx.x] = v;
        }
        __syncthreads();
    }
}

// Psi[q][j] = beta sum_i Phi[i][j] T[i][q] + alpha[j] V[q][j]: one thread per
// column j, NA_QB2 columns q per block row of the grid.
__global__ __launch_bounds__(128) void k_na_psi(const float* __restrict__ phi, long long N, long long D, long long ld,
                                                const float* __restrict__ T, int Q, const float* __restrict__ V,
                                                const float* __restrict__ alpha, float beta, float* __restrict__ Psi) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = blockIdx.y * NA_QB2;
    if (j >= D) return;
    float acc[NA_QB2];
#pragma unroll
    for (int k = 0; k < NA_QB2; ++k) acc[k] = 0.0f;
    for (long long i = 0; i < N; ++i) {
        const float a = phi[i * ld + j];
        const float* Ti = T + i * Q + q0;
#pragma unroll
        for (int k = 0; k < NA_QB2; ++k)
            if (q0 + k < Q) acc[k] = fmaf(a, Ti[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < NA_QB2; ++k)
        if (q0 + k < Q) {
            const size_t idx = (size_t)(q0 + k) * D + j;
            Psi[idx] = beta * acc[k] + alpha[j] * V[idx];
        }
}

}  // namespace

extern "C" cofem_status cofem_apply_dense_noalloc(const float* phi, long long N, long long D, long long ld,
                                                  const float* V, int Q, const float* alpha, double beta,
                                                  float* Psi, void* stream) {
    if (!phi || !V || !alpha || !Psi) return cofem_set_error(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (N < 1 || D < 1 || ld < D || N > 0x7fffffffLL || D > 0x7fffffffLL)
        return cofem_set_error(COFEM_ERR_INVALID_ARG, "need N, D >= 1 and ld >= D");
    if (Q < 1 || Q > COFEM_QMAX) return cofem_set_error(COFEM_ERR_INVALID_ARG, "need 1 <= Q <= 64");
    if ((unsigned long long)N * (unsigned long long)Q > (unsigned long long)COFEM_NOALLOC_MAX_ELEMS) {
        char msg[200];
        snprintf(msg, sizeof(msg), "N*Q = %lld exceeds the static scratch of %d floats", N * (long long)Q,
                 COFEM_NOALLOC_MAX_ELEMS);
        return cofem_set_error(COFEM_ERR_INVALID_ARG, msg);
    }
    if (!(beta == beta) || beta - beta != 0.0) return cofem_set_error(COFEM_ERR_NONFINITE, "beta is not finite");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cofem_set_error(COFEM_ERR_CUDA, cudaGetErrorString(e));
    if (!is_device_memory(phi, dev) || !is_device_memory(V, dev) || !is_device_memory(alpha, dev) ||
        !is_device_memory(Psi, dev))
        return cofem_set_error(COFEM_ERR_INVALID_ARG,
                               "phi, V, alpha and Psi must be device memory of the current device");
    float* T = nullptr;
    cofem_status st = na_scratch(dev, &T);
    if (st) return st;
    // an error left by an earlier, unrelated launch on this thread is reported
    // as such, not as a failure of these launches
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "a CUDA error was pending before this call: %s", cudaGetErrorString(e));
        return cofem_set_error(COFEM_ERR_CUDA, msg);
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_na_phiv<<<(unsigned)N, 256, 0, s>>>(phi, N, D, ld, V, Q, T);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cofem_set_error(COFEM_ERR_CUDA, cudaGetErrorString(e));
    const dim3 grid2((unsigned)((D + 127) / 128), (unsigned)((Q + NA_QB2 - 1) / NA_QB2));
    k_na_psi<<<grid2, 128, 0, s>>>(phi, N, D, ld, T, Q, V, alpha, (float)beta, Psi);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cofem_set_error(COFEM_ERR_CUDA, cudaGetErrorString(e));
    return COFEM_OK;
}
