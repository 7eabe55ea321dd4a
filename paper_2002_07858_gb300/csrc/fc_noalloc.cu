// fc_noalloc.cu -- fake-data generation that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need fake data:
// callers that run inside another framework's allocator hook or callback
// (which may not re-enter the allocator), and services that forbid device
// allocation on their request path after start-up (an allocation can stall
// on the device or fail under memory pressure).  For them
// fc_fake_data_noalloc produces exactly the output of fc_fake_data while its
// only scratch memory (the per-point systematic Cholesky factors and a status
// word) lives in the file-scope array below.
//
// The array is a fixed kNoAllocScratchBytes on every device that loads the
// library and stays resident until the process exits.  Every call shares it
// and it keeps the last call's contents; the status word is cleared at the
// start of each call.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "fc.h"
#include "fc_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;
constexpr int kDevBadCollapse = 8;  // status bit of k_check_collapse

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device (the host-side symbol is only
// a stand-in and must never be handed to a kernel).
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

fc_status noalloc_fail(fc_status st, const char* msg) {
    fcdev::record_error(msg);
    return st;
}

__global__ void k_check_points(const int64_t* __restrict__ ps, int P, int64_t G, int* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P && (ps[i] < 0 || ps[i] >= G)) atomicOr(status, fcdev::kDevBadIndex);
}

// The caller's collapse map (device memory, so it is checked on the device): every
// entry in [0, N_fit) and every fit bin reached by at least one full bin, the
// rules fc_load_grid applies on the host.  One CTA.
__global__ void k_check_collapse(const int32_t* __restrict__ coll, int nf, int nfit, int* __restrict__ status) {
    __shared__ int seen[fcdev::kMaxBins];
    for (int j = threadIdx.x; j < nfit; j += blockDim.x) seen[j] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const int32_t v = coll[i];
        if (v < 0 || v >= nfit)
            atomicOr(status, kDevBadCollapse);
        else
            seen[v] = 1;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nfit; j += blockDim.x)
        if (!seen[j]) atomicOr(status, kDevBadCollapse);
}

}  // namespace

extern "C" {

fc_status fc_fake_data_noalloc(const double* S, int64_t G, int32_t N_full, const int32_t* collapse, int32_t N_fit,
                               const double* F, const int64_t* ps, int32_t P, uint64_t seed, int32_t U,
                               int32_t fluct, float* d, void* cuda_stream) {
    if (!S || !F || !ps || !d) return noalloc_fail(FC_ERR_ARG, "NULL argument");
    if (G < 1 || N_full < 1 || N_full > fcdev::kMaxBins || N_fit < 1 || N_fit > fcdev::kMaxBins || P < 0 || U < 0)
        return noalloc_fail(FC_ERR_ARG, "sizes out of range");
    if (!collapse && N_fit != N_full) return noalloc_fail(FC_ERR_ARG, "N_fit must equal N_full without collapse");
    if (fluct != FC_FLUCT_POISSON_SYS && fluct != FC_FLUCT_GAUSS) return noalloc_fail(FC_ERR_ARG, "bad fluct");
    if (P == 0 || U == 0) return FC_OK;
    const size_t nf2 = (size_t)N_full * N_full;
    const size_t need = 256 + (size_t)P * nf2 * (sizeof(double) + sizeof(float)) + (size_t)P * N_full * sizeof(float);
    if (need > kNoAllocScratchBytes)
        return noalloc_fail(FC_ERR_ARG, "P * N_full^2 exceeds the 16 MiB static scratch (need P*N_full^2*12 + "
                                        "P*N_full*4 + 256 bytes); split the points over several calls");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(FC_ERR_CUDA, "no current CUDA device");
    // set-up once per device, with that device current
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return noalloc_fail(FC_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        base = (unsigned char*)g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int* status = (int*)base;
    double* L64 = (double*)(base + 256);
    float* L32 = (float*)(L64 + (size_t)P * nf2);
    float* s32 = L32 + (size_t)P * nf2;
    auto read_status = [&](int* h) -> bool {
        return cudaMemcpyAsync(h, status, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
               cudaStreamSynchronize(st) == cudaSuccess;
    };
    // the status word is the only state that must start at zero
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return noalloc_fail(FC_ERR_CUDA, "memset failed");
    // a launch error (bad configuration, no kernel image) is read before the call reports success
    auto launched = [&]() -> bool {
        const cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) return true;
        noalloc_fail(FC_ERR_CUDA, cudaGetErrorString(e));
        return false;
    };
    // validate the point indices and the collapse map before any kernel dereferences them
    fcdev::count_launch();
    k_check_points<<<(P + 255) / 256, 256, 0, st>>>(ps, P, G, status);
    if (!launched()) return FC_ERR_CUDA;
    if (collapse) {
        fcdev::count_launch();
        k_check_collapse<<<1, 256, 0, st>>>(collapse, N_full, N_fit, status);
        if (!launched()) return FC_ERR_CUDA;
    }
    int h = 0;
    if (!read_status(&h)) return noalloc_fail(FC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (h & fcdev::kDevBadIndex) return noalloc_fail(FC_ERR_ARG, "true point index out of range");
    if (h & kDevBadCollapse)
        return noalloc_fail(FC_ERR_ARG, "collapse map entry out of [0, N_fit) or a fit bin left empty");
    fcdev::launch_chol_sys(fcdev::FullSrc{S, {}}, N_full, F, ps, P, fluct == FC_FLUCT_GAUSS, L64, L32, s32, nullptr, status, st);
    if (!launched()) return FC_ERR_CUDA;
    fcdev::launch_fake_data(L32, s32, N_full, collapse, N_fit, ps, P, U, seed, fluct == FC_FLUCT_GAUSS, d, st);
    if (!launched()) return FC_ERR_CUDA;
    if (!read_status(&h)) return noalloc_fail(FC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (h & fcdev::kDevNotSpd) return noalloc_fail(FC_ERR_NOT_SPD, "systematic covariance not positive definite");
    return FC_OK;
}

}  // extern "C"
