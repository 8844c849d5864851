// vlbm_invariants_noalloc: the invariant reduction of vlbm_invariants, for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc/cudaFree are not available or
// not allowed -- inside a memory pool or arena that owns all device memory of
// the process, in a real-time loop that may not take the allocator's locks or
// its implicit device synchronisation, or close to the memory limit where an
// allocation could fail at an arbitrary point.  Such a caller owns the
// population lattice and the 8-double result; this entry point needs no
// handle, so it allocates nothing at all: the per-block FP64 partial sums live
// in the file-scope array below, which every GPU that loads the library keeps
// until the process exits ((8192 + 128 + 1) x 8 doubles, about 520 KiB).  One
// block reduces 8192 nodes, so lattices of up to 8192 x 8192 = 67,108,864 nodes
// are accepted; larger ones get VLBM_EINVAL.  Above 256 partial rows the rows
// are first folded by 128 blocks into 128 rows of the same array (as the
// handle's reduction does), so that the FP64 additions spread over many SMs.
// The lattice and a device `out` must be memory of the current device.
//
// Host code must not pass the array's name to a kernel: on the host that name
// is only a stand-in, not a device address.  The device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// cached; the first call on each device does that set-up, so make that first
// call before any stream capture.  Every call shares the array and finds the
// previous call's partials in it; each call writes every slot it later reads,
// so nothing needs clearing.  Calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "vlbm.h"
#include "vlbm_kernels_2d.cuh"
#include "vlbm_host.hpp"
#include "vlbm_fields.cuh"

using namespace vlbm;

namespace {

constexpr int kNoAllocMaxBlocks = 8192;           // partial rows
constexpr int kNoAllocStageRows = 128;            // first-stage rows when many partial rows are folded
constexpr int kNodesPerThread = 32;               // grid: one block per kThreads * 32 nodes
constexpr long long kNodesPerBlock = (long long)kThreads * kNodesPerThread;
constexpr int kMaxDevices = 64;

// Layout: kNoAllocMaxBlocks partial rows, kNoAllocStageRows first-stage rows, one
// row for a result bound for host memory; 8 doubles per row.
static __device__ __align__(256) double g_noalloc_partials[(kNoAllocMaxBlocks + kNoAllocStageRows + 1) * 8];

std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device (set-up on first use).
cudaError_t partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_ptr[dev] = static_cast<double*>(ptr);
    }
    *out = g_partials_ptr[dev];
    return cudaSuccess;
}

template <class C>
Coef<C> reduction_coef(const vlbm_params& p) {
    double scale[4];
    vlbm_storage_scales(p, scale);
    Coef<C> k{};
    for (int f = 0; f < kMaxFields; ++f) {
        k.scale[f] = (C)scale[f];
        k.inv_scale[f] = (C)(1.0 / scale[f]);
    }
    k.rho_bar = (C)p.rho_bar;
    return k;
}

template <class S, bool M>
void launch_partials(const vlbm_params& p, const void* lattice, long long nodes, int blocks, double* partials,
                     cudaStream_t s) {
    using C = typename Storage<S>::C;
    const Coef<C> k = reduction_coef<C>(p);
    if (p.dim == 2)
        k_invariants_2d<S, M><<<blocks, kThreads, 0, s>>>((const char*)lattice, nodes, k, partials);
    else
        k_invariants_3d<S, M><<<blocks, kThreads, 0, s>>>((const char*)lattice, nodes, k, partials);
}

// Where a pointer lives: 1 device memory of device `dev` (or managed memory),
// 0 host memory, -1 device memory of another device or an unknown pointer.
// A failed query's error is cleared here (it concerns only this query).
int pointer_home(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
}

}  // namespace

extern "C" int vlbm_invariants_noalloc(const vlbm_params* p, const void* lattice, double* out, void* stream) {
    if (!p || !lattice || !out) return VLBM_EINVAL;
    vlbm_derived d;
    if (vlbm_params_check(p, &d) < 0) return VLBM_EINVAL;
    const long long nodes = d.nodes;
    const long long blocks = (nodes + kNodesPerBlock - 1) / kNodesPerBlock;
    if (blocks > kNoAllocMaxBlocks) return VLBM_EINVAL;   // more than kNoAllocMaxBlocks * 8192 nodes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VLBM_ECUDA;
    if (pointer_home(lattice, dev) != 1) return VLBM_EINVAL;   // device memory of the current device only
    const int out_home = pointer_home(out, dev);
    if (out_home < 0) return VLBM_EINVAL;                      // another device's memory
    const bool out_on_device = out_home == 1;
    // an error left by the caller's earlier work is reported, not swallowed
    if (cudaPeekAtLastError() != cudaSuccess) return VLBM_ECUDA;
    double* partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) return VLBM_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    switch (p->precision) {
        case VLBM_FP64: launch_partials<double, false>(*p, lattice, nodes, (int)blocks, partials, s); break;
        case VLBM_FP32: launch_partials<float, false>(*p, lattice, nodes, (int)blocks, partials, s); break;
        case VLBM_FP16_SHIFTED: launch_partials<__half, false>(*p, lattice, nodes, (int)blocks, partials, s); break;
        case VLBM_BF16_SHIFTED:
            launch_partials<__nv_bfloat16, false>(*p, lattice, nodes, (int)blocks, partials, s);
            break;
        case VLBM_FP16_SPLIT: launch_partials<__half, true>(*p, lattice, nodes, (int)blocks, partials, s); break;
        default: launch_partials<__nv_bfloat16, true>(*p, lattice, nodes, (int)blocks, partials, s); break;
    }
    const double* rows = partials;
    int nrows = (int)blocks;
    if (nrows > 2 * kNoAllocStageRows) {   // fold the rows over many SMs first
        double* stage = partials + (size_t)kNoAllocMaxBlocks * 8;
        k_invariants_stage<<<kNoAllocStageRows, 256, 0, s>>>(partials, nrows, stage);
        rows = stage;
        nrows = kNoAllocStageRows;
    }
    // the last row holds the result when `out` is host memory
    double* result = out_on_device ? out : partials + (size_t)(kNoAllocMaxBlocks + kNoAllocStageRows) * 8;
    const double scale_e = p->dim == 3 ? p->dx : 1.0;
    k_invariants_final<<<1, 1024, 0, s>>>(rows, nrows, result, (double)nodes, p->rho_bar, 1.0 / p->dx, scale_e);
    if (cudaGetLastError() != cudaSuccess) return VLBM_ECUDA;
    if (!out_on_device) {
        if (cudaMemcpyAsync(out, result, 8 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return VLBM_ECUDA;
    }
    return VLBM_OK;
}
