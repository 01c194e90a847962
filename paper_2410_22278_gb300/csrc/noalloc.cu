// jk_energy_noalloc: the energy reduction of jk_energy with its scratch in a
// fixed file-scope device array, so that the call allocates no device memory.
//
// Who needs it: a caller whose device memory is owned by its own pool
// allocator under a fixed budget (a foreign cudaMalloc can fail there or
// fragment the pool), and a caller in a latency-bound loop that must not pay
// for an allocation or a free inside the library, which can synchronise the
// whole device.
//
// Scratch: kEnergyBlocks first-pass partials (two doubles each) and the two
// final sums, 64 KB in all, held by every device the library is loaded on
// until the process exits.  The first pass writes every partial that the
// second pass reads, so nothing has to start at zero and nothing is cleared.
// The array is shared by all calls on a device: two calls whose kernels
// overlap on the GPU (different streams or host threads) race on it.
//
// First call on a device: the array's device address is looked up once,
// with cudaGetSymbolAddress on that device; make that first call before any
// stream capture begins.  The address is kept for the life of the process:
// it assumes the device's primary context outlives the library's use of it
// (a cudaDeviceReset, or any other replacement of the primary context,
// invalidates it; such a program must not call this entry point again).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "plan.h"

namespace jk {
namespace {

constexpr int kEnergyThreads = 256;
constexpr int kEnergyBlocks = 4096;                  // most first-pass blocks
constexpr long long kEnergyMinPerBlock = 4096;       // fewest elements a block sums
constexpr long long kEnergyMaxPerBlock = 1LL << 16;  // most elements a block sums
// largest matrix: n^2 <= kEnergyBlocks * kEnergyMaxPerBlock, i.e. nbf <= 16384
constexpr long long kEnergyMaxElems = (long long)kEnergyBlocks * kEnergyMaxPerBlock;
constexpr int kEnergyMaxNbf = 16384;

static __device__ __align__(256) double g_energy_scratch[2 * kEnergyBlocks + 2];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;
}

// First pass: block b sums D.J and D.K over elements [b*per_block,
// (b+1)*per_block) and writes both partials unconditionally.
__global__ void k_energy_partials(long long n2, long long per_block, const double *__restrict__ D, const double *__restrict__ J,
                                  const double *__restrict__ K, double *__restrict__ scratch)
{
    __shared__ double sh[32];
    const long long lo = (long long)blockIdx.x * per_block;
    const long long hi = lo + per_block < n2 ? lo + per_block : n2;
    double sj = 0, sk = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double d = D[i];
        if (J) sj += d * J[i];
        if (K) sk += d * K[i];
    }
    sj = block_sum(sj, sh);
    sk = block_sum(sk, sh);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = sj;
        scratch[2 * blockIdx.x + 1] = sk;
    }
}

// Second pass: one block adds the nblk partials and scales them to E_J and E_K.
__global__ void k_energy_final(int nblk, double *__restrict__ scratch)
{
    __shared__ double sh[32];
    double sj = 0, sk = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        sj += scratch[2 * b];
        sk += scratch[2 * b + 1];
    }
    sj = block_sum(sj, sh);
    sk = block_sum(sk, sh);
    if (threadIdx.x == 0) {
        scratch[2 * kEnergyBlocks] = 0.5 * sj;
        scratch[2 * kEnergyBlocks + 1] = -0.25 * sk;
    }
}

int scratch_on_device(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(JK_ERR_INVALID, "jk_energy_noalloc: device index above 63");
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_energy_scratch);
        if (e != cudaSuccess || !p)
            return fail(JK_ERR_CUDA, std::string("jk_energy_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return JK_OK;
}

}  // namespace

int energy_noalloc(const Plan *P, const double *D, const double *J, const double *K, double *e_coul, double *e_exch,
                   cudaStream_t st)
{
    const long long n2 = (long long)P->nbf * P->nbf;
    if (P->nbf > kEnergyMaxNbf || n2 > kEnergyMaxElems)
        return fail(JK_ERR_INVALID, "jk_energy_noalloc: nbf = " + std::to_string(P->nbf) +
                                        " is above its fixed-scratch limit of 16384 basis functions (use jk_energy)");
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(JK_ERR_CUDA, "jk_energy_noalloc: cudaSetDevice failed");
    double *scratch = nullptr;
    const int rc = scratch_on_device(P->device, &scratch);
    if (rc) return rc;
    const long long per_block = std::max(kEnergyMinPerBlock, (n2 + kEnergyBlocks - 1) / kEnergyBlocks);
    const int nblk = (int)std::max(1LL, (n2 + per_block - 1) / per_block);  // <= kEnergyBlocks
    k_energy_partials<<<nblk, kEnergyThreads, 0, st>>>(n2, per_block, D, J, K, scratch);
    k_energy_final<<<1, kEnergyThreads, 0, st>>>(nblk, scratch);
    if (cudaGetLastError() != cudaSuccess) return fail(JK_ERR_CUDA, "jk_energy_noalloc: launch failed");
    double h[2] = {0, 0};
    if (cudaMemcpyAsync(h, scratch + 2 * kEnergyBlocks, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail(JK_ERR_CUDA, "jk_energy_noalloc: copy of the result failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(JK_ERR_CUDA, "jk_energy_noalloc: reduction failed");
    *e_coul = h[0];
    *e_exch = h[1];
    return JK_OK;
}

}  // namespace jk
