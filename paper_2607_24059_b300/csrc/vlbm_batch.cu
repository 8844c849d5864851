// Batched execution: many independent periodic 2D problems (each with its own
// size, dx, viscosity and time step dx^2/mu) advanced together, one persistent
// launch per time step over a work list of (problem, row, row segment) items,
// the launches of a run replayed from a captured CUDA graph.
//
// Every problem keeps the storage of a single handle (same kernels, same
// arithmetic: the per-warp step bodies of vlbm_kernels_2d.cuh / vlbm_split.cuh),
// at its own offset in one allocation per time level.  A step of the batch is a
// step of every problem; kernel boundaries order the steps, so no kernel waits
// on another.  Work items are numbered problem by problem, row by row.  The launch shape (threads per block, blocks per SM, nodes per
// lane of the split kernels) is chosen by vlbm_batch_autotune, which times each
// candidate on dry-run steps that read the current level and write the other
// one without committing it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vlbm.h"
#include "vlbm_host.hpp"
#include "vlbm_split.cuh"
#include "vlbm_fields.cuh"

using namespace vlbm;

namespace {

constexpr int kBatchGraphSteps = 32;   // steps per captured graph (even)
constexpr int kMaxBatchThreads = 256;

// One problem as the step kernel sees it.
template <class C>
struct BatchProblem {
    long long offset;        // bytes from the level base
    long long plane;         // nodes
    long long item0;         // first work item of this problem
    int nx, ny, wpr;         // sizes, warps (row segments) per row
    int vec;                 // 1: n_x is a multiple of the vector width (the vectorised warp body);
                             // 0: one node per lane, 32 per row segment (the per-node body)
    FastDiv wdiv;            // division by wpr
    Coef<C> k;
};

// One time step of every problem.  Warps take items in the strided order
// item = warp, warp + nwarps, ...: at any moment the grid works on a contiguous
// band of rows, so the rows y -+ 1 one warp reads were just read by another and
// come from L2.  The owning problem comes from the chunk table (problem of item
// 64 c) and at most a few forward steps.
constexpr int kChunkShift = 6;

// At most 128 registers (two 256-thread blocks per SM): the split body of the single lattice fits
// them without spilling; unbounded, the compiler took 146-149 and one block ran per SM.  The
// shifted 16-bit storage moves half the bytes of FP32 per node, so a warp has few bytes in
// flight unless it requests every load of its lane before the first shuffle (kLoadFirst, as the
// single-lattice kernel does).  Measured at 512 problems, FP16 shifted: interleaved 78 GLUPS,
// load-first at 128 registers 90 GLUPS, load-first bounded to 80 registers (three blocks per SM,
// ~130 bytes of spills) 86 GLUPS.  FP32 keeps the interleaved order (load-first: 50.5 against 53.0).
template <class S, bool SPLIT, int V = 4> struct BatchShape {
    static constexpr bool kLoadFirst = sizeof(S) == 2 && !SPLIT;
    // two nodes per lane halve the registers of the load-first body: three 256-thread blocks per SM
    static constexpr int kMinBlocks = (kLoadFirst && V == 2) ? 3 : 2;
};

template <class S, bool SPLIT, int V>
__global__ void __launch_bounds__(kMaxBatchThreads, (BatchShape<S, SPLIT, V>::kMinBlocks))
k_batch_step_2d(const char* __restrict__ in_base, char* __restrict__ out_base,
                const BatchProblem<typename Storage<S>::C>* __restrict__ probs, const int* __restrict__ chunk_problem,
                int count, long long items, uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // one step counter for the batch; nodes are numbered within their problem, so
    // a problem's rounding matches a single handle's at the same step
    const uint32_t key = take_step_key(step_ctr, par);
    Acc<C> unused;
    for (long long item = warp; item < items; item += nwarps) {   // warp-uniform
        int p = __ldg(chunk_problem + (item >> kChunkShift));
        while (p + 1 < count && probs[p + 1].item0 <= item) ++p;
        const BatchProblem<C>& P = probs[p];
        const long long local = item - P.item0;
        const uint32_t y = P.wdiv.div((uint32_t)local);
        const int seg = (int)((uint32_t)local - y * (uint32_t)P.wpr);
        const Layout<S, SPLIT, 5> fin{const_cast<char*>(in_base) + P.offset, P.plane};
        const Layout<S, SPLIT, 5> fout{out_base + P.offset, P.plane};
        const Coef<C>& k = P.k;   // read through L1, not copied into registers
        if (!P.vec) {             // warp-uniform: one node per lane
            const int x = seg * 32 + lane;
            const long long node = (long long)y * P.nx + x;
            if (x < P.nx) {
                if constexpr (SPLIT) node_split_step_2d<S, false>(fin, fout, P.nx, P.ny, node, k, unused);
                else node_stream_collide_2d<S, SPLIT, false>(fin, fout, P.nx, P.ny, node, k, unused, key);
            }
        } else if constexpr (SPLIT) {
            warp_split_step_2d<S, V, false>(fin, fout, P.nx, P.ny, (int)y, seg, lane, k, unused);
        } else {
            warp_stream_collide_2d<S, false, V, BatchShape<S, SPLIT>::kLoadFirst>(
                                             reinterpret_cast<const S*>(in_base + P.offset),
                                             reinterpret_cast<S*>(out_base + P.offset), P.plane, P.nx, P.ny, (int)y, seg,
                                             lane, k, unused, key);
        }
    }
}

// Grid-wide barrier of a cooperative launch (every block resident): block counts arrive on
// *count, which the host zeroes before the launch; barrier k completes when it reaches
// (k + 1) * gridDim.x.  The wait is bounded (about one second of globaltimer), and a block
// that gives up, or sees another block's failure in *status, records it and returns false.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int target, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned long long t0 = global_ns();
        int ok = 1;
        while (ld_acquire_gpu(count) < target) {
            if (*(volatile int*)status != 0 || global_ns() - t0 > 1000000000ull) {
                ok = 0;
                atomicExch(status, 1);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// nsteps time steps of every problem in one cooperative launch (VLBM_STEP_PERSISTENT): the
// body of k_batch_step_2d per step, levels alternating from par0, a grid barrier between steps.
// A step reads what the previous step of other blocks wrote, so its lattice loads are the
// coherent L2 loads (COH) instead of the read-only path.  The step counter of the stochastic
// rounding advances in registers; block 0 leaves step0 + nsteps in the slot the next launch reads.
template <class S, bool SPLIT, int V>
__global__ void __launch_bounds__(kMaxBatchThreads, (BatchShape<S, SPLIT, V>::kMinBlocks))
k_batch_steps_2d(char* level0, char* level1, const BatchProblem<typename Storage<S>::C>* __restrict__ probs,
                 const int* __restrict__ chunk_problem, int count, long long items, uint32_t* step_ctr, int par0,
                 int nsteps, unsigned int* bar_count, int* status, unsigned int phantom) {
    using C = typename Storage<S>::C;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint32_t step0 = __ldcg(step_ctr + par0);
    Acc<C> unused;
    for (int s = 0; s < nsteps; ++s) {
        const int par = (par0 + s) & 1;
        const char* in_base = par ? level1 : level0;
        char* out_base = par ? level0 : level1;
        const uint32_t key = sr_step_key(step0 + (uint32_t)s);
        for (long long item = warp; item < items; item += nwarps) {   // warp-uniform
            int p = __ldg(chunk_problem + (item >> kChunkShift));
            while (p + 1 < count && probs[p + 1].item0 <= item) ++p;
            const BatchProblem<C>& P = probs[p];
            const long long local = item - P.item0;
            const uint32_t y = P.wdiv.div((uint32_t)local);
            const int seg = (int)((uint32_t)local - y * (uint32_t)P.wpr);
            const Layout<S, SPLIT, 5> fin{const_cast<char*>(in_base) + P.offset, P.plane};
            const Layout<S, SPLIT, 5> fout{out_base + P.offset, P.plane};
            const Coef<C>& k = P.k;
            if (!P.vec) {
                const int x = seg * 32 + lane;
                const long long node = (long long)y * P.nx + x;
                if (x < P.nx) {
                    if constexpr (SPLIT) node_split_step_2d<S, false, true>(fin, fout, P.nx, P.ny, node, k, unused);
                    else node_stream_collide_2d<S, SPLIT, false, true>(fin, fout, P.nx, P.ny, node, k, unused, key);
                }
            } else if constexpr (SPLIT) {
                warp_split_step_2d<S, V, false, true>(fin, fout, P.nx, P.ny, (int)y, seg, lane, k, unused);
            } else {
                warp_stream_collide_2d<S, false, V, BatchShape<S, SPLIT>::kLoadFirst, true>(
                    reinterpret_cast<const S*>(in_base + P.offset), reinterpret_cast<S*>(out_base + P.offset), P.plane,
                    P.nx, P.ny, (int)y, seg, lane, k, unused, key);
            }
        }
        // (phantom = 1 only in the test of the timeout path: a block that never arrives)
        if (s + 1 < nsteps && !grid_barrier(bar_count, (unsigned int)(s + 1) * gridDim.x + phantom, status)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) step_ctr[(par0 + nsteps) & 1] = step0 + (uint32_t)nsteps;
}

// Masked initialisation / read-out of equally sized problems against one state
// array states [count][channels][ny][nx] FP32: channels 0, 1 = u, channel 2 =
// phi when channels >= 3.  blockIdx.y = problem; problems with mask 0 are skipped.
template <class S, bool SPLIT>
__global__ void __launch_bounds__(kThreads)
k_batch_init_states(char* __restrict__ level, const BatchProblem<typename Storage<S>::C>* __restrict__ probs,
                    const float* __restrict__ states, int channels, const uint8_t* __restrict__ mask, double dx,
                    double gamma, double rho_bar, double p_bar) {
    const int p = blockIdx.y;
    if (!mask[p]) return;
    const BatchProblem<typename Storage<S>::C>& P = probs[p];
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= P.plane) return;
    const float* st = states + (long long)p * channels * P.plane;
    init_node_2d<S, SPLIT, float>(Layout<S, SPLIT, 5>{level + P.offset, P.plane}, P.plane, node, st,
                                  channels > 2 ? st + 2 * P.plane : nullptr, P.k, dx, gamma, rho_bar, p_bar);
}

// The read-out writes FP32.  With FP32 (or 16-bit) storage the five populations of a moment are
// summed in FP32 with error-free transformations (Knuth's TwoSum; the compensated sum is as
// accurate as an FP64 sum rounded to FP32, also when the populations cancel), and the divisions
// by dx rho and dx^2 rho_bar are FP32 (a correctly rounded reciprocal times the moment, about
// 1.5 ulp): the FP64 form of these sums and divisions runs on the GPU's slow FP64 pipe.
template <class S, bool SPLIT>
__global__ void __launch_bounds__(kThreads)
k_batch_macros_states(const char* __restrict__ level, const BatchProblem<typename Storage<S>::C>* __restrict__ probs,
                      float* __restrict__ states, int channels, const uint8_t* __restrict__ mask, double dx,
                      double gamma, double rho_bar, double p_bar) {
    const int p = blockIdx.y;
    if (!mask[p]) return;
    const BatchProblem<typename Storage<S>::C>& P = probs[p];
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= P.plane) return;
    float* st = states + (long long)p * channels * P.plane;
    const Layout<S, SPLIT, 5> f{const_cast<char*>(level) + P.offset, P.plane};
    using C = typename Storage<S>::C;
    if constexpr (sizeof(C) == 8) {
        macros_node_2d<S, SPLIT, float>(f, P.plane, node, nullptr, st, channels > 2 ? st + 2 * P.plane : nullptr,
                                        P.k, dx, gamma, rho_bar, p_bar);
    } else {
        float m[3];
#pragma unroll
        for (int fld = 0; fld < 3; ++fld) {
            if constexpr (SPLIT) {
                m[fld] = f.rest(fld)[node];
            } else {
                float sum = load_pop(f, fld, 0, node, P.k), err = 0.0f;
#pragma unroll
                for (int l = 1; l < 5; ++l) {
                    const float x = load_pop(f, fld, l, node, P.k);
                    const float t = __fadd_rn(sum, x), bp = __fsub_rn(t, sum);
                    err = __fadd_rn(err, __fadd_rn(__fsub_rn(sum, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
                    sum = t;
                }
                m[fld] = __fadd_rn(sum, err);
            }
        }
        const float inv = 1.0f / ((float)dx * ((float)rho_bar + m[0]));
        st[node] = m[1] * inv;
        st[P.plane + node] = m[2] * inv;
        if (channels > 2) {
            const float dP = (gamma == 1.0) ? m[0] : (float)p_bar * expm1f((float)gamma * log1pf(m[0] / (float)rho_bar));
            st[2 * P.plane + node] = dP * (1.0f / (float)(dx * dx * rho_bar));
        }
    }
}

}  // namespace

struct vlbm_batch {
    std::vector<vlbm_params> p;
    std::vector<vlbm_derived> d;
    std::vector<long long> offset;
    int precision = VLBM_FP32;
    int count = 0;
    int sm_count = 148;
    cudaStream_t stream = nullptr;
    char* level[2] = {nullptr, nullptr};
    size_t level_bytes = 0;
    int cur = 0;
    void* table = nullptr;          // BatchProblem<C>[count] on the device
    uint32_t* ctr = nullptr;        // step counter of the stochastic rounding (2 slots, see take_step_key),
                                    // then the persistent launch's barrier count and status word
    int* status_host = nullptr;     // pinned copy of the status word
    int* chunks = nullptr;          // problem of item 64 c, c = 0 .. items / 64
    long long items = 0;
    int threads = 256, blocks_per_sm = 4, lanes = 4;
    double* partials = nullptr;
    int partial_blocks = 0;
    double* inv_dev = nullptr;
    double* inv_host = nullptr;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t step = 0, launches = 0;
    std::string err;
};

namespace {

int bfail(vlbm_batch* b, int code, const char* what, cudaError_t e) {
    if (b) b->err = std::string(what) + ": " + cudaGetErrorString(e);
    return code;
}

#define VLBM_BCUDA(b, call)                                                                              \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return bfail((b), e_ == cudaErrorMemoryAllocation ? VLBM_ENOMEM : VLBM_ECUDA, \
                                            #call, e_);                                                  \
    } while (0)

// Formats whose nodes per lane are a launch-shape choice (2 or 4, vlbm_batch_set_config): the
// split layouts and the shifted 16-bit storage.
bool lanes_tunable(int precision) {
    return is_split(precision) || precision == VLBM_FP16_SHIFTED || precision == VLBM_BF16_SHIFTED;
}

// Nodes per lane of the step kernel for the batch's precision and config.
int batch_lanes(const vlbm_batch* b) {
    if (lanes_tunable(b->precision)) return b->lanes;
    switch (b->precision) {
        case VLBM_FP64: return Vec16<double>::V;
        case VLBM_FP32: return Vec16<float>::V;
        default: return Vec16<__half>::V;
    }
}

template <class C>
int upload_table(vlbm_batch* b) {
    const int V = batch_lanes(b);
    std::vector<BatchProblem<C>> t(b->count);
    long long item = 0;
    for (int i = 0; i < b->count; ++i) {
        double scale[4];
        vlbm_storage_scales(b->p[i], scale);
        t[i].offset = b->offset[i];
        t[i].plane = b->d[i].nodes;
        t[i].nx = (int)b->p[i].n[0];
        t[i].ny = (int)b->p[i].n[1];
        t[i].vec = b->p[i].n[0] % V == 0;
        t[i].wpr = (int)(t[i].vec ? (b->p[i].n[0] / V + 31) / 32 : (b->p[i].n[0] + 31) / 32);
        t[i].wdiv = FastDiv::make((uint32_t)t[i].wpr);
        t[i].item0 = item;
        t[i].k = make_coef<C>(b->p[i], b->d[i], scale);
        item += (long long)t[i].ny * t[i].wpr;
    }
    b->items = item;
    std::vector<int> chunk((size_t)((item >> kChunkShift) + 1), 0);
    for (int i = 0, c = 0; c < (int)chunk.size(); ++c) {
        const long long first = (long long)c << kChunkShift;
        while (i + 1 < b->count && t[i + 1].item0 <= first) ++i;
        chunk[c] = i;
    }
    if (!b->table) VLBM_BCUDA(b, cudaMalloc(&b->table, sizeof(BatchProblem<C>) * b->count));
    if (b->chunks) {
        VLBM_BCUDA(b, cudaStreamSynchronize(b->stream));
        cudaFree(b->chunks);
        b->chunks = nullptr;
    }
    VLBM_BCUDA(b, cudaMalloc(&b->chunks, sizeof(int) * chunk.size()));
    VLBM_BCUDA(b, cudaMemcpyAsync(b->table, t.data(), sizeof(BatchProblem<C>) * b->count, cudaMemcpyHostToDevice,
                                  b->stream));
    VLBM_BCUDA(b, cudaMemcpyAsync(b->chunks, chunk.data(), sizeof(int) * chunk.size(), cudaMemcpyHostToDevice,
                                  b->stream));
    VLBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    return VLBM_OK;
}

int rebuild_table(vlbm_batch* b) {
    return b->precision == VLBM_FP64 ? upload_table<double>(b) : upload_table<float>(b);
}

void drop_graphs(vlbm_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

template <class S, bool SPLIT, int V>
void launch_batch(vlbm_batch* b, cudaStream_t s, int src) {
    using C = typename Storage<S>::C;
    k_batch_step_2d<S, SPLIT, V><<<b->sm_count * b->blocks_per_sm, b->threads, 0, s>>>(
        b->level[src], b->level[src ^ 1], (const BatchProblem<C>*)b->table, b->chunks, b->count, b->items, b->ctr,
        src);
}

void launch_batch_step(vlbm_batch* b, cudaStream_t s, int src) {
    switch (b->precision) {
        case VLBM_FP64: launch_batch<double, false, Vec16<double>::V>(b, s, src); break;
        case VLBM_FP32: launch_batch<float, false, Vec16<float>::V>(b, s, src); break;
        case VLBM_FP16_SHIFTED:
            if (b->lanes == 2) launch_batch<__half, false, 2>(b, s, src);
            else launch_batch<__half, false, 4>(b, s, src);
            break;
        case VLBM_BF16_SHIFTED:
            if (b->lanes == 2) launch_batch<__nv_bfloat16, false, 2>(b, s, src);
            else launch_batch<__nv_bfloat16, false, 4>(b, s, src);
            break;
        case VLBM_FP16_SPLIT:
            if (b->lanes == 2) launch_batch<__half, true, 2>(b, s, src);
            else launch_batch<__half, true, 4>(b, s, src);
            break;
        default:
            if (b->lanes == 2) launch_batch<__nv_bfloat16, true, 2>(b, s, src);
            else launch_batch<__nv_bfloat16, true, 4>(b, s, src);
            break;
    }
}

// One cooperative launch of k_batch_steps_2d for nsteps steps: the launch shape of the per-step
// kernel, its grid capped at the blocks that can be resident together.
template <class S, bool SPLIT, int V>
int launch_batch_steps(vlbm_batch* b, int nsteps, unsigned int phantom) {
    using C = typename Storage<S>::C;
    auto kernel = k_batch_steps_2d<S, SPLIT, V>;
    int per_sm = 0;
    VLBM_BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, b->threads, 0));
    if (per_sm < 1) return VLBM_EINVAL;
    const int grid = b->sm_count * std::min(per_sm, b->blocks_per_sm);
    char* l0 = b->level[0];
    char* l1 = b->level[1];
    const BatchProblem<C>* probs = (const BatchProblem<C>*)b->table;
    const int* chunks = b->chunks;
    int count = b->count;
    long long items = b->items;
    uint32_t* ctr = b->ctr;
    int par0 = b->cur;
    unsigned int* bar = reinterpret_cast<unsigned int*>(b->ctr + 2);
    int* status = reinterpret_cast<int*>(b->ctr + 3);
    void* args[] = {&l0, &l1, &probs, &chunks, &count, &items, &ctr, &par0, &nsteps, &bar, &status, &phantom};
    VLBM_BCUDA(b, cudaMemsetAsync(b->ctr + 2, 0, 2 * sizeof(uint32_t), b->stream));
    VLBM_BCUDA(b, cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(b->threads), args, 0, b->stream));
    return VLBM_OK;
}

int launch_batch_steps_any(vlbm_batch* b, int nsteps, unsigned int phantom) {
    switch (b->precision) {
        case VLBM_FP64: return launch_batch_steps<double, false, Vec16<double>::V>(b, nsteps, phantom);
        case VLBM_FP32: return launch_batch_steps<float, false, Vec16<float>::V>(b, nsteps, phantom);
        case VLBM_FP16_SHIFTED:
            return b->lanes == 2 ? launch_batch_steps<__half, false, 2>(b, nsteps, phantom)
                                 : launch_batch_steps<__half, false, 4>(b, nsteps, phantom);
        case VLBM_BF16_SHIFTED:
            return b->lanes == 2 ? launch_batch_steps<__nv_bfloat16, false, 2>(b, nsteps, phantom)
                                 : launch_batch_steps<__nv_bfloat16, false, 4>(b, nsteps, phantom);
        case VLBM_FP16_SPLIT:
            return b->lanes == 2 ? launch_batch_steps<__half, true, 2>(b, nsteps, phantom)
                                 : launch_batch_steps<__half, true, 4>(b, nsteps, phantom);
        default:
            return b->lanes == 2 ? launch_batch_steps<__nv_bfloat16, true, 2>(b, nsteps, phantom)
                                 : launch_batch_steps<__nv_bfloat16, true, 4>(b, nsteps, phantom);
    }
}

bool device_pointer(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ensure_bstaging(vlbm_batch* b, size_t bytes) {
    if (b->staging_bytes >= bytes) return VLBM_OK;
    if (b->staging) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->staging);
        b->staging = nullptr;
        b->staging_bytes = 0;
    }
    VLBM_BCUDA(b, cudaMalloc(&b->staging, bytes));
    b->staging_bytes = bytes;
    return VLBM_OK;
}

void free_batch(vlbm_batch* b) {
    drop_graphs(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (int i = 0; i < 2; ++i)
        if (b->level[i]) cudaFree(b->level[i]);
    if (b->table) cudaFree(b->table);
    if (b->ctr) cudaFree(b->ctr);
    if (b->chunks) cudaFree(b->chunks);
    if (b->partials) cudaFree(b->partials);
    if (b->inv_dev) cudaFree(b->inv_dev);
    if (b->inv_host) cudaFreeHost(b->inv_host);
    if (b->status_host) cudaFreeHost(b->status_host);
    if (b->staging) cudaFree(b->staging);
}

// Per-problem kernels reuse the single-lattice ones on the problem's slice.
template <class S, bool SPLIT, class T>
void launch_problem_init(vlbm_batch* b, int i, const T* u, const T* phi) {
    using C = typename Storage<S>::C;
    double scale[4];
    vlbm_storage_scales(b->p[i], scale);
    const Coef<C> k = make_coef<C>(b->p[i], b->d[i], scale);
    const long long N = b->d[i].nodes;
    k_init_2d<S, SPLIT, T><<<(N + kThreads - 1) / kThreads, kThreads, 0, b->stream>>>(
        b->level[b->cur] + b->offset[i], N, u, phi, k, b->p[i].dx, b->p[i].gamma, b->p[i].rho_bar,
        std::pow(b->p[i].rho_bar, b->p[i].gamma));
}

template <class S, bool SPLIT, class T>
void launch_problem_macros(vlbm_batch* b, int i, T* rho, T* u, T* phi) {
    using C = typename Storage<S>::C;
    double scale[4];
    vlbm_storage_scales(b->p[i], scale);
    const Coef<C> k = make_coef<C>(b->p[i], b->d[i], scale);
    const long long N = b->d[i].nodes;
    k_macros_2d<S, SPLIT, T><<<(N + kThreads - 1) / kThreads, kThreads, 0, b->stream>>>(
        b->level[b->cur] + b->offset[i], N, rho, u, phi, k, b->p[i].dx, b->p[i].gamma, b->p[i].rho_bar,
        std::pow(b->p[i].rho_bar, b->p[i].gamma));
}

template <class S, bool SPLIT>
void launch_problem_invariants(vlbm_batch* b, int i) {
    using C = typename Storage<S>::C;
    double scale[4];
    vlbm_storage_scales(b->p[i], scale);
    const Coef<C> k = make_coef<C>(b->p[i], b->d[i], scale);
    k_invariants_2d<S, SPLIT><<<b->partial_blocks, kThreads, 0, b->stream>>>(b->level[b->cur] + b->offset[i],
                                                                             b->d[i].nodes, k, b->partials);
    k_invariants_final<<<1, 1024, 0, b->stream>>>(b->partials, b->partial_blocks, b->inv_dev, (double)b->d[i].nodes,
                                                   b->p[i].rho_bar, 1.0 / b->p[i].dx, 1.0);
}

#define VLBM_BATCH_DISPATCH(b, FN, ...)                                            \
    switch ((b)->precision) {                                                      \
        case VLBM_FP64: FN<double, false>(__VA_ARGS__); break;                     \
        case VLBM_FP32: FN<float, false>(__VA_ARGS__); break;                      \
        case VLBM_FP16_SHIFTED: FN<__half, false>(__VA_ARGS__); break;             \
        case VLBM_BF16_SHIFTED: FN<__nv_bfloat16, false>(__VA_ARGS__); break;      \
        case VLBM_FP16_SPLIT: FN<__half, true>(__VA_ARGS__); break;                \
        default: FN<__nv_bfloat16, true>(__VA_ARGS__); break;                      \
    }

template <class S, bool SPLIT>
void init_any(vlbm_batch* b, int i, const void* u, const void* phi, int dtype) {
    if (dtype == VLBM_DTYPE_F64) launch_problem_init<S, SPLIT, double>(b, i, (const double*)u, (const double*)phi);
    else launch_problem_init<S, SPLIT, float>(b, i, (const float*)u, (const float*)phi);
}

template <class S, bool SPLIT>
void macros_any(vlbm_batch* b, int i, void* rho, void* u, void* phi, int dtype) {
    if (dtype == VLBM_DTYPE_F64) launch_problem_macros<S, SPLIT, double>(b, i, (double*)rho, (double*)u, (double*)phi);
    else launch_problem_macros<S, SPLIT, float>(b, i, (float*)rho, (float*)u, (float*)phi);
}

int build_batch_graph(vlbm_batch* b, int src) {
    if (!b->capture_stream) VLBM_BCUDA(b, cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    VLBM_BCUDA(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    int l = src;
    for (int i = 0; i < kBatchGraphSteps; ++i) {
        launch_batch_step(b, b->capture_stream, l);
        l ^= 1;
    }
    cudaGraph_t g = nullptr;
    VLBM_BCUDA(b, cudaStreamEndCapture(b->capture_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->graph[src], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph[src] = nullptr;
        return bfail(b, VLBM_ECUDA, "graph instantiate", e);
    }
    return VLBM_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" int vlbm_batch_create(const vlbm_params* problems, int32_t count, void* stream, vlbm_batch** out) {
    if (!out || !problems || count < 1) return VLBM_EINVAL;
    *out = nullptr;
    const int prec = problems[0].precision;
    std::vector<vlbm_derived> d(count);
    for (int i = 0; i < count; ++i) {
        const vlbm_params& q = problems[i];
        if (q.dim != 2 || q.precision != prec) return VLBM_EINVAL;
        if (q.n[0] > (1 << 24) || q.n[1] > (1 << 24)) return VLBM_EINVAL;
        if (vlbm_params_check(&q, &d[i]) < 0) return VLBM_EINVAL;
    }
    vlbm_batch* b = new (std::nothrow) vlbm_batch();
    if (!b) return VLBM_ENOMEM;
    b->p.assign(problems, problems + count);
    b->d = d;
    b->precision = prec;
    b->count = count;
    b->stream = (cudaStream_t)stream;
    size_t off = 0, largest = 0;
    for (int i = 0; i < count; ++i) {
        b->offset.push_back((long long)off);
        off += (d[i].lattice_bytes + 255) & ~(size_t)255;
        largest = std::max(largest, (size_t)d[i].nodes);
    }
    b->level_bytes = off;
    int dev = 0;
    int st = VLBM_OK;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        st = VLBM_ECUDA;
    for (int i = 0; i < 2 && st == VLBM_OK; ++i)
        if (cudaMalloc((void**)&b->level[i], off) != cudaSuccess) st = VLBM_ENOMEM;
    b->partial_blocks = (int)std::min<long long>(((long long)largest + kThreads - 1) / kThreads, b->sm_count * 8LL);
    if (st == VLBM_OK &&
        (cudaMalloc(&b->partials, (size_t)b->partial_blocks * 8 * sizeof(double)) != cudaSuccess ||
         cudaMalloc(&b->inv_dev, 8 * sizeof(double)) != cudaSuccess ||
         cudaMalloc(&b->ctr, 4 * sizeof(uint32_t)) != cudaSuccess ||
         cudaMallocHost(&b->inv_host, 8 * sizeof(double)) != cudaSuccess ||
         cudaMallocHost(&b->status_host, sizeof(int)) != cudaSuccess))
        st = VLBM_ENOMEM;
    if (st == VLBM_OK && (cudaMemsetAsync(b->level[0], 0, off, b->stream) != cudaSuccess ||
                          cudaMemsetAsync(b->ctr, 0, 4 * sizeof(uint32_t), b->stream) != cudaSuccess))
        st = VLBM_ECUDA;
    if (st == VLBM_OK) st = rebuild_table(b);
    if (st != VLBM_OK) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        return st;
    }
    *out = b;
    return VLBM_OK;
}

extern "C" void vlbm_batch_destroy(vlbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

extern "C" int vlbm_batch_init(vlbm_batch* b, int32_t problem, const void* u, const void* phi, int32_t dtype) {
    if (!b || !u || problem < 0 || problem >= b->count || (dtype != VLBM_DTYPE_F32 && dtype != VLBM_DTYPE_F64))
        return VLBM_EINVAL;
    const size_t es = dtype == VLBM_DTYPE_F64 ? 8 : 4;
    const long long N = b->d[problem].nodes;
    const size_t ub = 2 * N * es, pb = phi ? N * es : 0;
    const void* ud = u;
    const void* pd = phi;
    const bool host = !device_pointer(u) || (phi && !device_pointer(phi));
    if (host) {
        int rc = ensure_bstaging(b, ub + pb);
        if (rc) return rc;
        VLBM_BCUDA(b, cudaMemcpyAsync(b->staging, u, ub, cudaMemcpyDefault, b->stream));
        ud = b->staging;
        if (phi) {
            VLBM_BCUDA(b, cudaMemcpyAsync((char*)b->staging + ub, phi, pb, cudaMemcpyDefault, b->stream));
            pd = (char*)b->staging + ub;
        }
    }
    VLBM_BATCH_DISPATCH(b, init_any, b, problem, ud, pd, dtype);
    VLBM_BCUDA(b, cudaGetLastError());
    b->launches++;
    if (host) VLBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    return VLBM_OK;
}

extern "C" int vlbm_batch_step(vlbm_batch* b, int64_t nsteps, int32_t flags) {
    if (!b || nsteps < 0) return VLBM_EINVAL;
    if (flags & VLBM_STEP_PERSISTENT) {
        // all steps in cooperative launches of at most 2^30 steps, then the status word
        for (int64_t left = nsteps; left > 0;) {
            const int n = (int)std::min<int64_t>(left, 1 << 30);
            int rc = launch_batch_steps_any(b, n, (flags & VLBM_STEP_TEST_TIMEOUT) ? 1u : 0u);
            if (rc) return rc;
            b->launches++;
            b->step += n;
            if (n & 1) b->cur ^= 1;
            left -= n;
        }
        if (nsteps == 0) return VLBM_OK;
        VLBM_BCUDA(b, cudaMemcpyAsync(b->status_host, b->ctr + 3, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        VLBM_BCUDA(b, cudaStreamSynchronize(b->stream));
        if (*b->status_host != 0) {
            b->err = "a grid barrier of the persistent batched step gave up waiting";
            return VLBM_ETIMEOUT;
        }
        return VLBM_OK;
    }
    const bool graphs = !(flags & VLBM_STEP_NO_GRAPH);
    int64_t left = nsteps;
    while (left > 0) {
        if (graphs && left >= kBatchGraphSteps) {
            if (!b->graph[b->cur]) {
                int rc = build_batch_graph(b, b->cur);
                if (rc) return rc;
            }
            VLBM_BCUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
            b->launches += kBatchGraphSteps;
            b->step += kBatchGraphSteps;
            left -= kBatchGraphSteps;
        } else {
            launch_batch_step(b, b->stream, b->cur);
            VLBM_BCUDA(b, cudaGetLastError());
            b->launches++;
            b->cur ^= 1;
            b->step++;
            left--;
        }
    }
    return VLBM_OK;
}

extern "C" int vlbm_batch_macros(vlbm_batch* b, int32_t problem, void* rho, void* u, void* phi, int32_t dtype) {
    if (!b || problem < 0 || problem >= b->count || (dtype != VLBM_DTYPE_F32 && dtype != VLBM_DTYPE_F64))
        return VLBM_EINVAL;
    if (!rho && !u && !phi) return VLBM_OK;
    const size_t es = dtype == VLBM_DTYPE_F64 ? 8 : 4;
    const long long N = b->d[problem].nodes;
    void* out[3] = {rho, u, phi};
    const size_t bytes[3] = {N * es, 2 * N * es, N * es};
    void* dev[3] = {rho, u, phi};
    bool host[3] = {false, false, false};
    size_t off = 0, offs[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
        if (out[i] && !device_pointer(out[i])) {
            host[i] = true;
            offs[i] = off;
            off += bytes[i];
        }
    if (off) {
        int rc = ensure_bstaging(b, off);
        if (rc) return rc;
        for (int i = 0; i < 3; ++i)
            if (host[i]) dev[i] = (char*)b->staging + offs[i];
    }
    VLBM_BATCH_DISPATCH(b, macros_any, b, problem, dev[0], dev[1], dev[2], dtype);
    VLBM_BCUDA(b, cudaGetLastError());
    b->launches++;
    if (off) {
        for (int i = 0; i < 3; ++i)
            if (host[i]) VLBM_BCUDA(b, cudaMemcpyAsync(out[i], dev[i], bytes[i], cudaMemcpyDeviceToHost, b->stream));
        VLBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    }
    return VLBM_OK;
}

namespace {

// The masked state entry points need problems of one size and one dx, gamma, rho_bar.
bool uniform_problems(const vlbm_batch* b) {
    for (int i = 1; i < b->count; ++i) {
        const vlbm_params &a = b->p[0], &q = b->p[i];
        if (q.n[0] != a.n[0] || q.n[1] != a.n[1] || q.dx != a.dx || q.gamma != a.gamma || q.rho_bar != a.rho_bar)
            return false;
    }
    return true;
}

template <class S, bool SPLIT>
void launch_init_states(vlbm_batch* b, const float* states, int channels, const uint8_t* mask) {
    const vlbm_params& p = b->p[0];
    const dim3 grid((unsigned)((b->d[0].nodes + kThreads - 1) / kThreads), (unsigned)b->count);
    k_batch_init_states<S, SPLIT><<<grid, kThreads, 0, b->stream>>>(
        b->level[b->cur], (const BatchProblem<typename Storage<S>::C>*)b->table, states, channels, mask, p.dx,
        p.gamma, p.rho_bar, std::pow(p.rho_bar, p.gamma));
}

template <class S, bool SPLIT>
void launch_macros_states(vlbm_batch* b, float* states, int channels, const uint8_t* mask) {
    const vlbm_params& p = b->p[0];
    const dim3 grid((unsigned)((b->d[0].nodes + kThreads - 1) / kThreads), (unsigned)b->count);
    k_batch_macros_states<S, SPLIT><<<grid, kThreads, 0, b->stream>>>(
        b->level[b->cur], (const BatchProblem<typename Storage<S>::C>*)b->table, states, channels, mask, p.dx,
        p.gamma, p.rho_bar, std::pow(p.rho_bar, p.gamma));
}

}  // namespace

extern "C" int vlbm_batch_init_states(vlbm_batch* b, const float* states, int32_t channels, const uint8_t* mask) {
    if (!b || !states || !mask || channels < 2 || b->count > 65535) return VLBM_EINVAL;
    if (b->p[0].dim != 2 || !uniform_problems(b) || !device_pointer(states) || !device_pointer(mask))
        return VLBM_EINVAL;
    VLBM_BATCH_DISPATCH(b, launch_init_states, b, states, channels, mask);
    VLBM_BCUDA(b, cudaGetLastError());
    b->launches++;
    return VLBM_OK;
}

extern "C" int vlbm_batch_macros_states(vlbm_batch* b, float* states, int32_t channels, const uint8_t* mask) {
    if (!b || !states || !mask || channels < 2 || b->count > 65535) return VLBM_EINVAL;
    if (b->p[0].dim != 2 || !uniform_problems(b) || !device_pointer(states) || !device_pointer(mask))
        return VLBM_EINVAL;
    VLBM_BATCH_DISPATCH(b, launch_macros_states, b, states, channels, mask);
    VLBM_BCUDA(b, cudaGetLastError());
    b->launches++;
    return VLBM_OK;
}

extern "C" int vlbm_batch_invariants(vlbm_batch* b, int32_t problem, double* out) {
    if (!b || !out || problem < 0 || problem >= b->count) return VLBM_EINVAL;
    VLBM_BATCH_DISPATCH(b, launch_problem_invariants, b, problem);
    VLBM_BCUDA(b, cudaGetLastError());
    b->launches += 2;
    if (device_pointer(out)) {
        VLBM_BCUDA(b, cudaMemcpyAsync(out, b->inv_dev, 8 * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
        return VLBM_OK;
    }
    VLBM_BCUDA(b, cudaMemcpyAsync(b->inv_host, b->inv_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    VLBM_BCUDA(b, cudaStreamSynchronize(b->stream));
    std::memcpy(out, b->inv_host, 8 * sizeof(double));
    return VLBM_OK;
}

extern "C" int vlbm_batch_set_config(vlbm_batch* b, int32_t threads, int32_t blocks_per_sm, int32_t lanes) {
    if (!b || (threads != 128 && threads != 256) || blocks_per_sm < 1 || blocks_per_sm > 16) return VLBM_EINVAL;
    if (lanes_tunable(b->precision) && lanes != 2 && lanes != 4) return VLBM_EINVAL;
    const bool relayout = lanes_tunable(b->precision) && lanes != b->lanes;   // the work list depends on it
    b->threads = threads;
    b->blocks_per_sm = blocks_per_sm;
    if (lanes_tunable(b->precision)) b->lanes = lanes;
    drop_graphs(b);
    return relayout ? rebuild_table(b) : VLBM_OK;
}

extern "C" int vlbm_batch_autotune(vlbm_batch* b, int32_t repeats, int32_t* config_out, double* best_ms) {
    if (!b || repeats < 1) return VLBM_EINVAL;
    const int thread_opts[2] = {128, 256};
    const int bps_opts[5] = {1, 2, 4, 8, 16};
    const int lane_opts[2] = {2, 4};
    const int nl = lanes_tunable(b->precision) ? 2 : 1;
    cudaEvent_t e0, e1;
    VLBM_BCUDA(b, cudaEventCreate(&e0));
    VLBM_BCUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = b->threads, bb = b->blocks_per_sm, bl = b->lanes;
    int rc = VLBM_OK;
    for (int li = 0; li < nl && rc == VLBM_OK; ++li)
        for (int ti = 0; ti < 2 && rc == VLBM_OK; ++ti)
            for (int bi = 0; bi < 5 && rc == VLBM_OK; ++bi) {
                rc = vlbm_batch_set_config(b, thread_opts[ti], bps_opts[bi], nl > 1 ? lane_opts[li] : b->lanes);
                if (rc) break;
                // dry runs: read the current level, write the other, do not commit
                launch_batch_step(b, b->stream, b->cur);
                cudaEventRecord(e0, b->stream);
                for (int r = 0; r < repeats; ++r) launch_batch_step(b, b->stream, b->cur);
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                    rc = VLBM_ECUDA;
                    break;
                }
                b->launches += repeats + 1;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= repeats;
                if (ms < best) {
                    best = ms;
                    bt = b->threads;
                    bb = b->blocks_per_sm;
                    bl = b->lanes;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = vlbm_batch_set_config(b, bt, bb, bl);
    if (rc) return rc;
    if (config_out) {
        config_out[0] = bt;
        config_out[1] = bb;
        config_out[2] = bl;
    }
    if (best_ms) *best_ms = best;
    return VLBM_OK;
}

extern "C" int vlbm_batch_info(const vlbm_batch* b, int64_t* nodes_total, int64_t* step, int64_t* launches) {
    if (!b) return VLBM_EINVAL;
    if (nodes_total) {
        int64_t n = 0;
        for (const auto& d : b->d) n += d.nodes;
        *nodes_total = n;
    }
    if (step) *step = b->step;
    if (launches) *launches = b->launches;
    return VLBM_OK;
}

extern "C" const char* vlbm_batch_last_error(const vlbm_batch* b) { return b ? b->err.c_str() : "null batch"; }
