// C ABI of the vectorial lattice Boltzmann library (declared in include/vlbm.h).
// Host-side logic: parameter resolution (Section 2, Prop. 1, Lemmas 1-2),
// buffer ownership, launch configuration, CUDA-graph replay of step batches,
// host/device pointer staging and checkpoints.  Every step of the scheme runs
// in the kernels of vlbm_kernels_2d.cuh / vlbm_kernels_3d.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "vlbm.h"
#include "vlbm_kernels_2d.cuh"
#include "vlbm_kernels_3d.cuh"
#include "vlbm_split.cuh"
#include "vlbm_fields.cuh"
#include "vlbm_boundary.cuh"
#include "vlbm_host.hpp"

using namespace vlbm;

namespace {

// Steps captured per CUDA graph, largest first (even: a replay keeps the parity of the levels).
// Replays run each step about 6 us faster than single launches at 4096^2, so runs shorter than
// the largest graph replay the smaller ones too.
constexpr int kGraphSizes = 3;
constexpr int kGraphSteps[kGraphSizes] = {64, 16, 4};
constexpr int kStageBlocks = 128;             // first-stage blocks when many partial rows are reduced
constexpr uint64_t kStateMagic = 0x315F4D424C56ull;  // "VLBM_1"

struct StateHeader {
    uint64_t magic;
    int32_t dim, precision;
    int64_t n[3];
    int64_t step;
    uint64_t lattice_bytes;
    double dx, mu;
    double omega[4], alpha[4];
};

}  // namespace

struct vlbm_handle {
    vlbm_params p{};
    vlbm_derived d{};
    int device = 0;
    int sm_count = 148;
    cudaStream_t stream = nullptr;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    double* partials = nullptr;
    int64_t partial_capacity = 0;     // blocks
    double* stage = nullptr;          // kStageBlocks rows of the two-stage final reduction
    double* inv_dev = nullptr;        // 8 doubles
    uint32_t* ctr = nullptr;          // step counter of the stochastic rounding: ctr[cur] = step (mod 2^32)
    unsigned int* fold_ctr = nullptr; // kStageBlocks + 1 tickets of the fused-diagnostics fold (zero between launches)
    double* inv_host = nullptr;       // 8 doubles, pinned
    void* staging = nullptr;
    size_t staging_bytes = 0;
    double* hist = nullptr;           // device records of vlbm_step_record for host destinations
    int64_t hist_capacity = 0;        // records
    int64_t step = 0;
    int64_t launches = 0;
    int kernel_variant = 0;           // 0 auto, 1 generic, 2 vectorised
    int split_lanes = kSplitV2;       // nodes per lane of the 2D split kernel (2 or 4)
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph[kGraphSizes][2] = {};   // [size][parity of the starting level]
    std::string err;
    Coef<double> kd{};
    Coef<float> kf{};
    // boundary conditions (vlbm_set_boundary): periodic, or the channel of Section 6.2.1
    int bc_kind = VLBM_BC_PERIODIC;
    int bc_correction = 0;
    double bc_phi_out = 0.0;
    double* bc_u_in = nullptr;        // n_y inflow velocities
    void* bc_ghost = nullptr;         // 4 sides x 3 fields x n_ghost entering populations
    int bc_n_ghost = 0;
};

// ------------------------------------------------------------------ helpers
namespace {

template <class C> const Coef<C>& coef(const vlbm_handle* h);
template <> const Coef<double>& coef<double>(const vlbm_handle* h) { return h->kd; }
template <> const Coef<float>& coef<float>(const vlbm_handle* h) { return h->kf; }

int fail(vlbm_handle* h, int code, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

#define VLBM_CUDA(h, call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail((h), e_ == cudaErrorMemoryAllocation ? VLBM_ENOMEM : VLBM_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

int check_launch(vlbm_handle* h, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, VLBM_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return VLBM_OK;
}

bool is_device_pointer(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ------------------------------------------------------------------ parameters
extern "C" void vlbm_params_default(vlbm_params* p, int32_t dim, const int64_t* n, double dx, double nu,
                                    int32_t precision) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->dim = dim;
    p->precision = precision;
    for (int i = 0; i < 3; ++i) p->n[i] = (n && i < dim) ? n[i] : 1;
    p->dx = dx;
    p->mu = 8.0;                 // Section 6.1
    p->nu = nu;
    p->omega[0] = 6.0 / 5.0;     // Eq. params, middle pair
    p->alpha[0] = 3.0 / 40.0;
    for (int k = 1; k < 4; ++k) {
        p->omega[k] = 23.0 / 20.0;   // Section 6.1.3
        p->alpha[k] = -1.0;          // from nu (Prop. 1)
    }
    p->gamma = 1.0;
    p->rho_bar = 1.0;
}

extern "C" int vlbm_params_check(const vlbm_params* p, vlbm_derived* out) {
    if (!p) return VLBM_EINVAL;
    if (p->dim != 2 && p->dim != 3) return VLBM_EINVAL;
    if (p->reserved != 0) return VLBM_EINVAL;
    if (elem_bytes(p->precision) == 0) return VLBM_EINVAL;
    for (int i = 0; i < p->dim; ++i)
        if (p->n[i] < 1 || p->n[i] > (int64_t)1 << 30) return VLBM_EINVAL;
    if (!(p->dx > 0.0) || !(p->mu > 0.0) || !(p->rho_bar > 0.0) || !(p->gamma >= 1.0) || !(p->nu >= 0.0))
        return VLBM_EINVAL;
    if (!std::isfinite(p->dx) || !std::isfinite(p->mu) || !std::isfinite(p->gamma) || !std::isfinite(p->nu))
        return VLBM_EINVAL;
    vlbm_derived d{};
    const int F = p->dim + 1;
    const double a_max = p->dim == 2 ? 0.25 : 1.0 / 6.0;   // Lemma 1 (3D: rest weight 1 - 6 alpha >= 0)
    for (int k = 0; k < F; ++k) {
        const double om = p->omega[k];
        if (!(om > 0.0 && om < 2.0)) return VLBM_EINVAL;   // (0, 2]; 2 is inviscid (Prop. 1)
        double al = p->alpha[k];
        if (k > 0 && al < 0.0) al = p->nu / (2.0 * p->mu * (1.0 / om - 0.5));   // Prop. 1
        if (!(al >= 0.0 && al <= a_max)) return VLBM_EINVAL;
        d.alpha[k] = al;
        d.viscosity[k] = 2.0 * p->mu * al * (1.0 / om - 0.5);
    }
    d.dt = p->dx * p->dx / p->mu;
    double amin = d.alpha[1];
    for (int k = 2; k < F; ++k) amin = std::min(amin, d.alpha[k]);
    const double s = d.alpha[0] + amin;
    d.mu_min = s > 0.0 ? 1.0 / std::sqrt(s) : INFINITY;
    d.nodes = p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1);
    d.populations_per_node = F * (2 * p->dim + 1);
    d.bytes_per_population = elem_bytes(p->precision);
    d.lattice_bytes = (size_t)layout_bytes(d.bytes_per_population, is_split(p->precision), 2 * p->dim + 1, d.nodes);
    if (out) *out = d;
    if (p->mu < d.mu_min) return p->strict ? VLBM_ESTABILITY : VLBM_WSTABILITY;
    return VLBM_OK;
}

// ------------------------------------------------------------------ lifecycle
static int64_t blocks_for(int64_t threads) { return (threads + kThreads - 1) / kThreads; }

// Nodes per lane of the vectorised step kernels (Vec16 / Vec8 in the kernel
// headers): 2D min(4, 16 B / element), 3D min(2, 8 B / element).
static int vec_width(const vlbm_handle* h) {
    if (is_split(h->p.precision)) return h->p.dim == 2 ? h->split_lanes : kSplitV3;
    const int b = h->d.bytes_per_population;
    return h->p.dim == 2 ? std::min(4, 16 / b) : std::min(2, 8 / b);
}

static bool use_vec(const vlbm_handle* h) {
    if (h->kernel_variant == 1) return false;
    const int64_t nx = h->p.n[0], v = vec_width(h);
    const int64_t items = h->d.nodes / nx * ((nx / v + 31) / 32);     // warp work items (32-bit in the kernels)
    return nx % v == 0 && (h->p.dim == 2 || h->p.dim == 3) && items < (int64_t(1) << 32) &&
           h->d.nodes < (int64_t(1) << 32);     // 32-bit node offsets
}

// Nodes per lane of the vectorised step with fused diagnostics (DiagVec: 2 for 2D FP32).
static int diag_vec_width(const vlbm_handle* h) {
    return (h->p.dim == 2 && h->p.precision == VLBM_FP32) ? 2 : vec_width(h);
}

static int64_t step_blocks_v(const vlbm_handle* h, int v) {
    const int64_t nx = h->p.n[0];
    const int64_t rows = h->d.nodes / nx;
    if (use_vec(h)) {
        const int64_t wpr = (nx / v + 31) / 32;
        return (rows * wpr * 32 + kThreads - 1) / kThreads;
    }
    return blocks_for(h->d.nodes);
}

static int64_t inv_blocks(const vlbm_handle* h) {
    return std::min<int64_t>(blocks_for(h->d.nodes), (int64_t)h->sm_count * 8);
}

// Destroy every captured step graph (their kernel parameters changed, or the handle is closed).
static void drop_graphs(vlbm_handle* h) {
    for (auto& per_size : h->graph)
        for (auto& g : per_size)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

static void free_all(vlbm_handle* h) {
    drop_graphs(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (int i = 0; i < 2; ++i)
        if (h->buf[i]) cudaFree(h->buf[i]);
    if (h->partials) cudaFree(h->partials);
    if (h->stage) cudaFree(h->stage);
    if (h->inv_dev) cudaFree(h->inv_dev);
    if (h->ctr) cudaFree(h->ctr);
    if (h->fold_ctr) cudaFree(h->fold_ctr);
    if (h->inv_host) cudaFreeHost(h->inv_host);
    if (h->staging) cudaFree(h->staging);
    if (h->hist) cudaFree(h->hist);
    if (h->bc_u_in) cudaFree(h->bc_u_in);
    if (h->bc_ghost) cudaFree(h->bc_ghost);
}

static void storage_scales(const vlbm_params& p, const vlbm_derived& d, double* scale) {
    (void)d;
    vlbm_storage_scales(p, scale);
}

extern "C" int vlbm_create(const vlbm_params* p, void* stream, vlbm_handle** out) {
    if (!out) return VLBM_EINVAL;
    *out = nullptr;
    vlbm_derived d;
    const int rc = vlbm_params_check(p, &d);
    if (rc < 0) return rc;
    vlbm_handle* h = new (std::nothrow) vlbm_handle();
    if (!h) return VLBM_ENOMEM;
    h->p = *p;
    h->d = d;
    h->stream = (cudaStream_t)stream;
    int st = VLBM_OK;
    do {
        if (cudaGetDevice(&h->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
            st = fail(h, VLBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        for (int i = 0; i < 2 && st == VLBM_OK; ++i) {
            cudaError_t e = cudaMalloc(&h->buf[i], d.lattice_bytes);
            if (e != cudaSuccess) st = VLBM_ENOMEM;
        }
        if (st != VLBM_OK) break;
        // any step variant may be selected later (VLBM_OPT_*): size for the largest
        // grid, one thread per node or one lane per node (vector width 1)
        const int64_t rows = d.nodes / p->n[0];
        const int64_t widest = (rows * ((p->n[0] + 31) / 32) * 32 + kThreads - 1) / kThreads;
        h->partial_capacity = std::max({blocks_for(d.nodes), widest, inv_blocks(h)});
        if (cudaMalloc(&h->partials, (size_t)h->partial_capacity * 8 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->stage, (size_t)kStageBlocks * 8 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->inv_dev, 8 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->ctr, 2 * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&h->fold_ctr, (kStageBlocks + 1) * sizeof(unsigned int)) != cudaSuccess ||
            cudaMallocHost(&h->inv_host, 8 * sizeof(double)) != cudaSuccess) {
            st = VLBM_ENOMEM;
            break;
        }
        if (cudaMemsetAsync(h->buf[0], 0, d.lattice_bytes, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->ctr, 0, 2 * sizeof(uint32_t), h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->fold_ctr, 0, (kStageBlocks + 1) * sizeof(unsigned int), h->stream) != cudaSuccess) {
            st = VLBM_ECUDA;
            break;
        }
    } while (0);
    if (st != VLBM_OK) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return st;
    }
    double scale[4];
    storage_scales(h->p, h->d, scale);
    h->kd = make_coef<double>(h->p, h->d, scale);
    h->kf = make_coef<float>(h->p, h->d, scale);
    *out = h;
    return rc;   // VLBM_OK or VLBM_WSTABILITY
}

extern "C" void vlbm_destroy(vlbm_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

extern "C" int vlbm_set_stream(vlbm_handle* h, void* stream) {
    if (!h) return VLBM_EINVAL;
    h->stream = (cudaStream_t)stream;
    return VLBM_OK;
}

// ------------------------------------------------------------------ staging
static int ensure_staging(vlbm_handle* h, size_t bytes) {
    if (h->staging_bytes >= bytes) return VLBM_OK;
    if (h->staging) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->staging);
        h->staging = nullptr;
        h->staging_bytes = 0;
    }
    VLBM_CUDA(h, cudaMalloc(&h->staging, bytes));
    h->staging_bytes = bytes;
    return VLBM_OK;
}

// ------------------------------------------------------------------ init / macros
template <class S, bool M, class T>
static void launch_init(vlbm_handle* h, const T* u, const T* phi) {
    const int64_t N = h->d.nodes;
    const double pb = std::pow(h->p.rho_bar, h->p.gamma);
    const auto& k = coef<typename Storage<S>::C>(h);
    if (h->p.dim == 2)
        k_init_2d<S, M, T><<<blocks_for(N), kThreads, 0, h->stream>>>((char*)h->buf[h->cur], N, u, phi, k, h->p.dx,
                                                                   h->p.gamma, h->p.rho_bar, pb);
    else
        k_init_3d<S, M, T><<<blocks_for(N), kThreads, 0, h->stream>>>((char*)h->buf[h->cur], N, u, phi, k, h->p.dx,
                                                                   h->p.gamma, h->p.rho_bar, pb);
    h->launches++;
}

template <class S, bool M, class T>
static void launch_macros(vlbm_handle* h, T* rho, T* u, T* phi) {
    const int64_t N = h->d.nodes;
    const double pb = std::pow(h->p.rho_bar, h->p.gamma);
    const auto& k = coef<typename Storage<S>::C>(h);
    if (h->p.dim == 2)
        k_macros_2d<S, M, T><<<blocks_for(N), kThreads, 0, h->stream>>>((const char*)h->buf[h->cur], N, rho, u, phi, k,
                                                                     h->p.dx, h->p.gamma, h->p.rho_bar, pb);
    else
        k_macros_3d<S, M, T><<<blocks_for(N), kThreads, 0, h->stream>>>((const char*)h->buf[h->cur], N, rho, u, phi, k,
                                                                     h->p.dx, h->p.gamma, h->p.rho_bar, pb);
    h->launches++;
}

// Instantiate FN<storage, mixed layout> for the handle's precision.
#define VLBM_DISPATCH_STORAGE(h, FN, ...)                                      \
    switch ((h)->p.precision) {                                                \
        case VLBM_FP64: FN<double, false>(__VA_ARGS__); break;                 \
        case VLBM_FP32: FN<float, false>(__VA_ARGS__); break;                  \
        case VLBM_FP16_SHIFTED: FN<__half, false>(__VA_ARGS__); break;         \
        case VLBM_BF16_SHIFTED: FN<__nv_bfloat16, false>(__VA_ARGS__); break;  \
        case VLBM_FP16_SPLIT: FN<__half, true>(__VA_ARGS__); break;            \
        default: FN<__nv_bfloat16, true>(__VA_ARGS__); break;                  \
    }

template <class S, bool M>
static void init_dispatch(vlbm_handle* h, const void* u, const void* phi, int dtype) {
    if (dtype == VLBM_DTYPE_F64) launch_init<S, M, double>(h, (const double*)u, (const double*)phi);
    else launch_init<S, M, float>(h, (const float*)u, (const float*)phi);
}

template <class S, bool M>
static void macros_dispatch(vlbm_handle* h, void* rho, void* u, void* phi, int dtype) {
    if (dtype == VLBM_DTYPE_F64) launch_macros<S, M, double>(h, (double*)rho, (double*)u, (double*)phi);
    else launch_macros<S, M, float>(h, (float*)rho, (float*)u, (float*)phi);
}

extern "C" int vlbm_init(vlbm_handle* h, const void* u, const void* phi, int32_t dtype) {
    if (!h || !u || (dtype != VLBM_DTYPE_F32 && dtype != VLBM_DTYPE_F64)) return VLBM_EINVAL;
    const size_t es = dtype == VLBM_DTYPE_F64 ? 8 : 4;
    const int64_t N = h->d.nodes;
    const size_t ub = (size_t)h->p.dim * N * es, pb = phi ? (size_t)N * es : 0;
    const void* ud = u;
    const void* pd = phi;
    const bool u_host = !is_device_pointer(u), p_host = phi && !is_device_pointer(phi);
    if (u_host || p_host) {
        int rc = ensure_staging(h, ub + pb);
        if (rc) return rc;
        if (u_host) {
            VLBM_CUDA(h, cudaMemcpyAsync(h->staging, u, ub, cudaMemcpyHostToDevice, h->stream));
            ud = h->staging;
        }
        if (p_host) {
            VLBM_CUDA(h, cudaMemcpyAsync((char*)h->staging + ub, phi, pb, cudaMemcpyHostToDevice, h->stream));
            pd = (char*)h->staging + ub;
        }
    }
    VLBM_DISPATCH_STORAGE(h, init_dispatch, h, ud, pd, dtype);
    int rc = check_launch(h, "init");
    if (rc) return rc;
    h->step = 0;
    VLBM_CUDA(h, cudaMemsetAsync(h->ctr + h->cur, 0, sizeof(uint32_t), h->stream));
    if (u_host || p_host) VLBM_CUDA(h, cudaStreamSynchronize(h->stream));   // host arrays may be reused on return
    return VLBM_OK;
}

extern "C" int vlbm_macros(vlbm_handle* h, void* rho, void* u, void* phi, int32_t dtype) {
    if (!h || (dtype != VLBM_DTYPE_F32 && dtype != VLBM_DTYPE_F64)) return VLBM_EINVAL;
    if (!rho && !u && !phi) return VLBM_OK;
    const size_t es = dtype == VLBM_DTYPE_F64 ? 8 : 4;
    const int64_t N = h->d.nodes;
    const size_t sb = (size_t)N * es, ub = (size_t)h->p.dim * N * es;
    void* out[3] = {rho, u, phi};
    const size_t bytes[3] = {sb, ub, sb};
    void* dev[3] = {rho, u, phi};
    bool host[3] = {false, false, false};
    size_t off = 0, offs[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        if (out[i] && !is_device_pointer(out[i])) {
            host[i] = true;
            offs[i] = off;
            off += bytes[i];
        }
    }
    if (off) {
        int rc = ensure_staging(h, off);
        if (rc) return rc;
        for (int i = 0; i < 3; ++i)
            if (host[i]) dev[i] = (char*)h->staging + offs[i];
    }
    VLBM_DISPATCH_STORAGE(h, macros_dispatch, h, dev[0], dev[1], dev[2], dtype);
    int rc = check_launch(h, "macros");
    if (rc) return rc;
    if (off) {
        for (int i = 0; i < 3; ++i)
            if (host[i]) VLBM_CUDA(h, cudaMemcpyAsync(out[i], dev[i], bytes[i], cudaMemcpyDeviceToHost, h->stream));
        VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return VLBM_OK;
}

// ------------------------------------------------------------------ stepping
static DiagSink diag_sink(vlbm_handle* h, double* out, int nblocks);

// One step from buffer src.  Plain steps launch one warp per row segment (one thread per
// node for the per-node kernels).  Steps with fused diagnostics (DIAG, out = where the 8
// invariants go) launch a persistent grid of the kernel's resident blocks on every SM,
// each warp looping over segments and accumulating before one block reduction and the
// fold of DiagSink.
template <class S, bool M, bool DIAG>
static void launch_step_on(vlbm_handle* h, cudaStream_t s, int src, double* out) {
    using C = typename Storage<S>::C;
    const auto& k = coef<C>(h);
    const char* fin = (const char*)h->buf[src];
    char* fout = (char*)h->buf[src ^ 1];
    const int64_t nx = h->p.n[0], ny = h->p.n[1];
    const int64_t plane = h->d.nodes;
    const int v = DIAG ? diag_vec_width(h) : vec_width(h);
    const int64_t blocks = step_blocks_v(h, v);
    const int64_t nz = h->p.n[2];
    const bool vec = use_vec(h);
    const int wpr = (int)((nx / v + 31) / 32);
    auto go = [&](auto kernel, auto... args) {
        int64_t grid = blocks;
        DiagSink sink{};
        if constexpr (DIAG) {
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess) per_sm = 1;
            grid = std::min<int64_t>(blocks, (int64_t)h->sm_count * std::max(per_sm, 1));
            sink = diag_sink(h, out, (int)grid);
        }
        kernel<<<(unsigned)grid, kThreads, 0, s>>>(args..., sink, h->ctr, src);
    };
    if constexpr (M) {
        if (h->p.dim == 2) {
            if (vec && h->split_lanes == 2)
                go(k_split_step_2d_vec<S, 2, DIAG>, fin, fout, (int)nx, (int)ny, plane, FastDiv::make(wpr), k);
            else if (vec)
                go(k_split_step_2d_vec<S, 4, DIAG>, fin, fout, (int)nx, (int)ny, plane, FastDiv::make(wpr), k);
            else
                go(k_split_step_2d_generic<S, DIAG>, fin, fout, (int)nx, (int)ny, plane, k);
        } else {
            if (vec)
                go(k_split_step_3d_vec<S, DIAG>, split_planes<S, 7>(fin, fout, plane), (int)nx, (int)ny, (int)nz,
                   FastDiv::make(wpr), FastDiv::make((uint32_t)ny), k);
            else
                go(k_split_step_3d_generic<S, DIAG>, fin, fout, (int)nx, (int)ny, (int)nz, plane, k);
        }
    } else if (h->p.dim == 2) {
        if (vec)
            go(k_stream_collide_2d_vec<S, M, DIAG>, fin, fout, (int)nx, (int)ny, plane, FastDiv::make(wpr), k);
        else
            go(k_stream_collide_2d_generic<S, M, DIAG>, fin, fout, (int)nx, (int)ny, plane, k);
    } else {
        if (vec)
            go(k_stream_collide_3d_vec<S, M, DIAG>, fin, fout, (int)nx, (int)ny, (int)nz, plane, wpr, k);
        else
            go(k_stream_collide_3d_generic<S, M, DIAG>, fin, fout, (int)nx, (int)ny, (int)nz, plane, k);
    }
}

template <class S, bool M>
static void step_plain(vlbm_handle* h, cudaStream_t s, int src) { launch_step_on<S, M, false>(h, s, src, nullptr); }

template <class S, bool M>
static void step_diag(vlbm_handle* h, cudaStream_t s, int src, double* out) {
    launch_step_on<S, M, true>(h, s, src, out);
}

// The fused-diagnostics sink of a step launched with nblocks blocks whose invariants go to
// out (device, 8 doubles): groups of at least 32 partial rows, at most kStageBlocks groups.
static DiagSink diag_sink(vlbm_handle* h, double* out, int nblocks) {
    DiagSink k{};
    k.partials = h->partials;
    k.stage = h->stage;
    k.counters = h->fold_ctr;
    k.out = out;
    k.nblocks = nblocks;
    k.group = std::max<int>(32, (nblocks + kStageBlocks - 1) / kStageBlocks);
    k.ngroups = (nblocks + k.group - 1) / k.group;
    k.nodes = (double)h->d.nodes;
    k.rho_bar = h->p.rho_bar;
    k.inv_dx = 1.0 / h->p.dx;
    k.scale_e = h->p.dim == 3 ? h->p.dx : 1.0;
    return k;
}

// One step of a channel (vlbm_set_boundary): the ghost populations of the four sides from the
// current level, then the per-node step that reads them where a pull crosses a side.
template <class S>
static void step_channel(vlbm_handle* h, cudaStream_t s, int src) {
    using C = typename Storage<S>::C;
    const int nx = (int)h->p.n[0], ny = (int)h->p.n[1];
    ChannelBC<C> bc;
    bc.u_in = h->bc_u_in;
    bc.ghost = (C*)h->bc_ghost;
    bc.n_ghost = h->bc_n_ghost;
    bc.phi_term = (C)(2.0 * h->p.rho_bar * h->p.dx * h->p.dx * h->bc_phi_out);
    bc.u_scale = (C)(2.0 * h->p.rho_bar * h->p.dx);
    bc.correction = h->bc_correction;
    const char* fin = (const char*)h->buf[src];
    k_channel_ghosts<S><<<dim3((unsigned)((h->bc_n_ghost + kThreads - 1) / kThreads), 4), kThreads, 0, s>>>(
        fin, nx, ny, h->d.nodes, coef<C>(h), bc);
    k_stream_collide_2d_channel<S><<<(unsigned)((h->d.nodes + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        fin, (char*)h->buf[src ^ 1], nx, ny, h->d.nodes, coef<C>(h), bc, h->ctr, src);
}

// Kernel launches of one step.
static int launches_per_step(const vlbm_handle* h) { return h->bc_kind == VLBM_BC_CHANNEL ? 2 : 1; }

static void dispatch_step(vlbm_handle* h, cudaStream_t s, int src) {
    if (h->bc_kind == VLBM_BC_CHANNEL) {
        if (h->p.precision == VLBM_FP64) step_channel<double>(h, s, src);
        else step_channel<float>(h, s, src);
        return;
    }
    VLBM_DISPATCH_STORAGE(h, step_plain, h, s, src);
}

static int launch_one_step(vlbm_handle* h, cudaStream_t s, int src) {
    dispatch_step(h, s, src);
    return check_launch(h, "stream-collide");
}

// Capture kGraphSteps[size] steps starting from buffer `src` on a private stream.
static int build_graph(vlbm_handle* h, int size, int src) {
    if (!h->capture_stream) VLBM_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    VLBM_CUDA(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    int b = src;
    int rc = VLBM_OK;
    for (int i = 0; i < kGraphSteps[size]; ++i) {
        dispatch_step(h, h->capture_stream, b);
        b ^= 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
    if (e != cudaSuccess) return fail(h, VLBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph[size][src], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph[size][src] = nullptr;
        rc = fail(h, VLBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return rc;
}

static int launch_invariants(vlbm_handle* h, double* out_dev);

extern "C" int vlbm_step(vlbm_handle* h, int64_t nsteps, int32_t flags) {
    if (!h || nsteps < 0) return VLBM_EINVAL;
    int64_t left = nsteps;
    const bool graphs = !(flags & VLBM_STEP_NO_GRAPH);
    while (left > 0) {
        int size = 0;
        while (size < kGraphSizes && left < kGraphSteps[size]) ++size;
        if (graphs && size < kGraphSizes) {
            if (!h->graph[size][h->cur]) {
                int rc = build_graph(h, size, h->cur);
                if (rc) return rc;
            }
            VLBM_CUDA(h, cudaGraphLaunch(h->graph[size][h->cur], h->stream));
            h->launches += (int64_t)kGraphSteps[size] * launches_per_step(h);
            h->step += kGraphSteps[size];
            left -= kGraphSteps[size];   // an even count: parity unchanged
        } else {
            int rc = launch_one_step(h, h->stream, h->cur);
            if (rc) return rc;
            h->launches += launches_per_step(h);
            h->cur ^= 1;
            h->step++;
            left--;
        }
    }
    if (flags & VLBM_STEP_CHECK_FINITE) {
        int rc = launch_invariants(h, h->inv_dev);
        if (rc) return rc;
        VLBM_CUDA(h, cudaMemcpyAsync(h->inv_host, h->inv_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->inv_host[6] != 0.0) return fail(h, VLBM_EDIVERGED, "%.0f non-finite nodes at step %lld", h->inv_host[6],
                                               (long long)h->step);
    }
    return VLBM_OK;
}

extern "C" int vlbm_set_boundary(vlbm_handle* h, const vlbm_boundary* bc) {
    if (!h || !bc) return VLBM_EINVAL;
    if (bc->kind == VLBM_BC_PERIODIC) {
        if (h->bc_kind != VLBM_BC_PERIODIC) {
            drop_graphs(h);
        }
        h->bc_kind = VLBM_BC_PERIODIC;
        return VLBM_OK;
    }
    if (bc->kind != VLBM_BC_CHANNEL) return fail(h, VLBM_EINVAL, "unknown boundary kind %d", bc->kind);
    if (h->p.dim != 2 || (h->p.precision != VLBM_FP64 && h->p.precision != VLBM_FP32))
        return fail(h, VLBM_EINVAL, "channel boundaries: 2D lattices with FP64 or FP32 storage only");
    if (h->p.n[0] < 2 || h->p.n[1] < 2) return fail(h, VLBM_EINVAL, "channel boundaries need at least 2 x 2 nodes");
    if (!bc->u_in || !std::isfinite(bc->phi_out)) return fail(h, VLBM_EINVAL, "channel boundaries: u_in and a finite phi_out");
    const int ny = (int)h->p.n[1];
    for (int j = 0; j < ny; ++j)
        if (!std::isfinite(bc->u_in[j])) return fail(h, VLBM_EINVAL, "channel boundaries: u_in[%d] is not finite", j);
    const int n_ghost = (int)std::max(h->p.n[0], h->p.n[1]);
    const size_t es = h->p.precision == VLBM_FP64 ? sizeof(double) : sizeof(float);
    if (!h->bc_u_in) VLBM_CUDA(h, cudaMalloc(&h->bc_u_in, (size_t)ny * sizeof(double)));
    if (!h->bc_ghost) VLBM_CUDA(h, cudaMalloc(&h->bc_ghost, (size_t)4 * 3 * n_ghost * es));
    VLBM_CUDA(h, cudaMemcpyAsync(h->bc_u_in, bc->u_in, (size_t)ny * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->bc_kind = VLBM_BC_CHANNEL;
    h->bc_correction = bc->wall_correction ? 1 : 0;
    h->bc_phi_out = bc->phi_out;
    h->bc_n_ghost = n_ghost;
    return VLBM_OK;
}

static void launch_final(vlbm_handle* h, int nblocks, double* out_dev);

// Pointer kinds for outputs: device, pinned (page-locked) host, pageable host.
enum PtrKind { kDevice, kPinned, kPageable };

static PtrKind pointer_kind(const void* ptr, void** device_view = nullptr) {
    cudaPointerAttributes a;
    if (device_view) *device_view = nullptr;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return kPageable;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return kDevice;
    if (a.type == cudaMemoryTypeHost) {
        if (device_view) *device_view = a.devicePointer;   // page-locked memory mapped for the device
        return kPinned;
    }
    return kPageable;
}

extern "C" int vlbm_step_record(vlbm_handle* h, int64_t nsteps, int64_t every, double* history) {
    if (!h || nsteps < 0 || every < 1 || (nsteps > 0 && !history)) return VLBM_EINVAL;
    if (h->bc_kind != VLBM_BC_PERIODIC)
        return fail(h, VLBM_EINVAL, "fused records need periodic boundaries (use vlbm_step and vlbm_invariants)");
    if (nsteps == 0) return VLBM_OK;
    const int64_t records = (nsteps + every - 1) / every;
    void* mapped = nullptr;
    PtrKind kind = pointer_kind(history, &mapped);
    double* rec = history;
    if (kind == kPinned && mapped) {
        // page-locked host memory mapped into the device's address space: the step kernel's
        // final fold writes each record there itself, so no copy follows the step in the stream
        rec = static_cast<double*>(mapped);
        kind = kDevice;
    }
    if (kind != kDevice) {
        if (h->hist_capacity < records) {
            if (h->hist) {
                VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
                cudaFree(h->hist);
                h->hist = nullptr;
                h->hist_capacity = 0;
            }
            VLBM_CUDA(h, cudaMalloc(&h->hist, (size_t)records * 8 * sizeof(double)));
            h->hist_capacity = records;
        }
        rec = h->hist;
    }
    for (int64_t s = 0; s < nsteps;) {
        if (s % every == 0) {
            // one launch: the step, its invariants and their fold (DiagSink)
            VLBM_DISPATCH_STORAGE(h, step_diag, h, h->stream, h->cur, rec + (s / every) * 8);
            int rc = check_launch(h, "stream-collide (diagnostics)");
            if (rc) return rc;
            h->launches += 1;
            h->cur ^= 1;
            h->step++;
            ++s;
        } else {
            // plain steps up to the next record (graph replay when long enough)
            const int64_t run = std::min(nsteps - s, every - s % every);
            int rc = vlbm_step(h, run, 0);
            if (rc) return rc;
            s += run;
        }
    }
    if (kind != kDevice) {
        VLBM_CUDA(h, cudaMemcpyAsync(history, rec, (size_t)records * 8 * sizeof(double), cudaMemcpyDeviceToHost,
                                     h->stream));
        if (kind == kPageable) VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return VLBM_OK;
}

// ------------------------------------------------------------------ invariants
template <class S, bool M>
static void invariants_partials(vlbm_handle* h, int blocks) {
    using C = typename Storage<S>::C;
    const auto& k = coef<C>(h);
    if (h->p.dim == 2)
        k_invariants_2d<S, M><<<blocks, kThreads, 0, h->stream>>>((const char*)h->buf[h->cur], h->d.nodes, k,
                                                                   h->partials);
    else
        k_invariants_3d<S, M><<<blocks, kThreads, 0, h->stream>>>((const char*)h->buf[h->cur], h->d.nodes, k,
                                                                   h->partials);
}

static void launch_final(vlbm_handle* h, int nblocks, double* out_dev) {
    const double inv_dx = 1.0 / h->p.dx;
    const double scale_e = h->p.dim == 3 ? h->p.dx : 1.0;
    const double* rows = h->partials;
    if (nblocks > 2 * kStageBlocks) {     // two stages: spread the FP64 additions over many SMs
        k_invariants_stage<<<kStageBlocks, 256, 0, h->stream>>>(h->partials, nblocks, h->stage);
        h->launches++;
        rows = h->stage;
        nblocks = kStageBlocks;
    }
    k_invariants_final<<<1, 1024, 0, h->stream>>>(rows, nblocks, out_dev, (double)h->d.nodes, h->p.rho_bar,
                                                   inv_dx, scale_e);
}

static int launch_invariants(vlbm_handle* h, double* out_dev) {
    const int blocks = (int)inv_blocks(h);
    VLBM_DISPATCH_STORAGE(h, invariants_partials, h, blocks);
    int rc = check_launch(h, "invariants");
    if (rc) return rc;
    launch_final(h, blocks, out_dev);
    h->launches += 2;      // partials + final (a first stage, when used, counts itself)
    return check_launch(h, "invariants final");
}

extern "C" int vlbm_invariants(vlbm_handle* h, double* out) {
    if (!h || !out) return VLBM_EINVAL;
    if (is_device_pointer(out)) return launch_invariants(h, out);
    int rc = launch_invariants(h, h->inv_dev);
    if (rc) return rc;
    VLBM_CUDA(h, cudaMemcpyAsync(h->inv_host, h->inv_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    std::memcpy(out, h->inv_host, 8 * sizeof(double));
    return VLBM_OK;
}

// ------------------------------------------------------------------ vorticity
extern "C" int vlbm_vorticity_sq(vlbm_handle* h, double* out) {
    if (!h || !out) return VLBM_EINVAL;
    const int64_t N = h->d.nodes;
    const int dim = h->p.dim;
    int rc = ensure_staging(h, (size_t)dim * N * sizeof(float));
    if (rc) return rc;
    float* u = (float*)h->staging;
    VLBM_DISPATCH_STORAGE(h, macros_dispatch, h, nullptr, u, nullptr, VLBM_DTYPE_F32);
    rc = check_launch(h, "macros");
    if (rc) return rc;
    const int blocks = (int)inv_blocks(h);
    k_vorticity_sq<<<blocks, kThreads, 0, h->stream>>>(u, (int)h->p.n[0], (int)h->p.n[1],
                                                        dim == 3 ? (int)h->p.n[2] : 1, dim, h->partials);
    const double inv2dx = 0.5 / h->p.dx;
    const double scale = inv2dx * inv2dx * std::pow(h->p.dx, (double)dim);
    const bool dev = is_device_pointer(out);
    k_sum_rows<<<1, kThreads, 0, h->stream>>>(h->partials, blocks, scale, dev ? out : h->inv_dev);
    h->launches += 3;
    rc = check_launch(h, "vorticity");
    if (rc) return rc;
    if (!dev) {
        VLBM_CUDA(h, cudaMemcpyAsync(h->inv_host, h->inv_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
        *out = h->inv_host[0];
    }
    return VLBM_OK;
}

// ------------------------------------------------------------------ time / state
extern "C" int vlbm_time(const vlbm_handle* h, int64_t* step, double* t) {
    if (!h) return VLBM_EINVAL;
    if (step) *step = h->step;
    if (t) *t = (double)h->step * h->d.dt;
    return VLBM_OK;
}

extern "C" size_t vlbm_state_bytes(const vlbm_handle* h) {
    return h ? sizeof(StateHeader) + h->d.lattice_bytes : 0;
}

static StateHeader make_header(const vlbm_handle* h) {
    StateHeader s{};
    s.magic = kStateMagic;
    s.dim = h->p.dim;
    s.precision = h->p.precision;
    for (int i = 0; i < 3; ++i) s.n[i] = h->p.n[i];
    s.step = h->step;
    s.lattice_bytes = h->d.lattice_bytes;
    s.dx = h->p.dx;
    s.mu = h->p.mu;
    for (int k = 0; k < 4; ++k) {
        s.omega[k] = h->p.omega[k];
        s.alpha[k] = h->d.alpha[k];
    }
    return s;
}

extern "C" int vlbm_get_state(vlbm_handle* h, void* dst, size_t bytes) {
    if (!h || !dst || bytes < vlbm_state_bytes(h)) return VLBM_EINVAL;
    const StateHeader s = make_header(h);
    VLBM_CUDA(h, cudaMemcpyAsync(dst, &s, sizeof s, cudaMemcpyDefault, h->stream));
    VLBM_CUDA(h, cudaMemcpyAsync((char*)dst + sizeof s, h->buf[h->cur], h->d.lattice_bytes, cudaMemcpyDefault,
                                 h->stream));
    VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return VLBM_OK;
}

extern "C" int vlbm_set_state(vlbm_handle* h, const void* src, size_t bytes) {
    if (!h || !src || bytes < vlbm_state_bytes(h)) return VLBM_EINVAL;
    StateHeader s{};
    VLBM_CUDA(h, cudaMemcpyAsync(&s, src, sizeof s, cudaMemcpyDefault, h->stream));
    VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    const StateHeader mine = make_header(h);
    if (s.magic != kStateMagic || s.dim != mine.dim || s.precision != mine.precision ||
        s.lattice_bytes != mine.lattice_bytes || std::memcmp(s.n, mine.n, sizeof s.n) != 0 || s.dx != mine.dx ||
        s.mu != mine.mu || std::memcmp(s.omega, mine.omega, sizeof s.omega) != 0 ||
        std::memcmp(s.alpha, mine.alpha, sizeof s.alpha) != 0)
        return fail(h, VLBM_EINVAL, "checkpoint does not match this handle's configuration");
    VLBM_CUDA(h, cudaMemcpyAsync(h->buf[h->cur], (const char*)src + sizeof s, h->d.lattice_bytes, cudaMemcpyDefault,
                                 h->stream));
    const uint32_t ctr = (uint32_t)s.step;   // the stochastic rounding continues where the checkpoint left off
    VLBM_CUDA(h, cudaMemcpyAsync(h->ctr + h->cur, &ctr, sizeof ctr, cudaMemcpyHostToDevice, h->stream));
    VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->step = s.step;
    return VLBM_OK;
}

template <class S, bool M, class T>
static void launch_export(vlbm_handle* h, T* dst, int deviation) {
    using C = typename Storage<S>::C;
    const auto& k = coef<C>(h);
    const int q = 2 * h->p.dim + 1;
    const int64_t total = h->d.nodes * h->d.populations_per_node;
    const double f_rest = (1.0 - 2.0 * h->p.dim * h->d.alpha[0]) * h->p.rho_bar;
    const double f_move = h->d.alpha[0] * h->p.rho_bar;
    const double p_half = std::pow(h->p.rho_bar, h->p.gamma) / (2.0 * h->p.mu);
    if (q == 5)
        k_export<S, M, 5, T><<<blocks_for(total), kThreads, 0, h->stream>>>(
            (const char*)h->buf[h->cur], total, h->d.nodes, dst, k, f_rest, f_move, p_half, deviation);
    else
        k_export<S, M, 7, T><<<blocks_for(total), kThreads, 0, h->stream>>>(
            (const char*)h->buf[h->cur], total, h->d.nodes, dst, k, f_rest, f_move, p_half, deviation);
    h->launches++;
}

template <class S, bool M>
static void export_dispatch(vlbm_handle* h, void* dst, int dtype, int deviation) {
    if (dtype == VLBM_DTYPE_F64) launch_export<S, M, double>(h, (double*)dst, deviation);
    else launch_export<S, M, float>(h, (float*)dst, deviation);
}

extern "C" int vlbm_get_populations(vlbm_handle* h, void* dst, int32_t dtype, int32_t deviation) {
    if (!h || !dst || (dtype != VLBM_DTYPE_F32 && dtype != VLBM_DTYPE_F64)) return VLBM_EINVAL;
    const size_t bytes = (size_t)h->d.nodes * h->d.populations_per_node * (dtype == VLBM_DTYPE_F64 ? 8 : 4);
    const bool host = !is_device_pointer(dst);
    void* d = dst;
    if (host) {
        int rc = ensure_staging(h, bytes);
        if (rc) return rc;
        d = h->staging;
    }
    VLBM_DISPATCH_STORAGE(h, export_dispatch, h, d, dtype, deviation);
    int rc = check_launch(h, "export");
    if (rc) return rc;
    if (host) {
        VLBM_CUDA(h, cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, h->stream));
        VLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return VLBM_OK;
}

extern "C" int vlbm_launch_count(const vlbm_handle* h, int64_t* count) {
    if (!h || !count) return VLBM_EINVAL;
    *count = h->launches;
    return VLBM_OK;
}

extern "C" int vlbm_set_option(vlbm_handle* h, int32_t key, int64_t value) {
    if (!h) return VLBM_EINVAL;
    switch (key) {
        case VLBM_OPT_KERNEL:
            if (value < 0 || value > 2) return VLBM_EINVAL;
            if (value == 2 && h->p.n[0] % vec_width(h) != 0) return VLBM_EINVAL;
            h->kernel_variant = (int)value;
            drop_graphs(h);
            return VLBM_OK;
        case VLBM_OPT_ROUNDING_16:
            if (value != 0 && value != 1) return VLBM_EINVAL;
            if (h->p.precision != VLBM_FP16_SHIFTED && h->p.precision != VLBM_BF16_SHIFTED) return VLBM_EINVAL;
            h->kf.sr16 = (int)value;   // a kernel parameter: captured graphs are rebuilt
            drop_graphs(h);
            return VLBM_OK;
        case VLBM_OPT_SPLIT_LANES:
            if (value != 2 && value != 4) return VLBM_EINVAL;
            if (h->p.dim == 2 && h->p.n[0] % value != 0 && h->kernel_variant == 2) return VLBM_EINVAL;
            h->split_lanes = (int)value;
            drop_graphs(h);
            return VLBM_OK;
        default: return VLBM_EINVAL;
    }
}

extern "C" const char* vlbm_strerror(int code) {
    switch (code) {
        case VLBM_OK: return "ok";
        case VLBM_WSTABILITY: return "mu below the low-frequency stability bound (warning)";
        case VLBM_EINVAL: return "invalid argument";
        case VLBM_ESTABILITY: return "mu below the low-frequency stability bound";
        case VLBM_ENOMEM: return "out of memory";
        case VLBM_ECUDA: return "CUDA error";
        case VLBM_EDIVERGED: return "non-finite populations";
        case VLBM_ETIMEOUT: return "device wait timed out";
        case VLBM_EUNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" const char* vlbm_last_error(const vlbm_handle* h) { return h ? h->err.c_str() : "null handle"; }
