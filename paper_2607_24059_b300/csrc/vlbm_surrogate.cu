// Tensor-core (tcgen05) kernels of the learned surrogate: a BF16 GEMM core
// (D = A B^T, FP32 accumulation in tensor memory) that the convolution layers
// are built on.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "vlbm.h"
#include "vlbm_tc.cuh"

using namespace vlbm;

namespace {

constexpr int kTcThreads = 128;          // one warpgroup: TMEM lanes 0..127
constexpr int kKChunk = 64;              // K columns staged per round
constexpr long long kWaitPolls = 1 << 22;

// Kernels launched by this file's entry points since the library was loaded.
std::atomic<long long> g_launches{0};

// Device pointers the kernels access in vectors of `bytes` must be aligned to them.
bool misaligned(const void* p, uintptr_t bytes) { return reinterpret_cast<uintptr_t>(p) % bytes != 0; }

// D[M x N] = A[M x K] B[N x K]^T for one 128-row block of A.  A, B row-major
// BF16 (K contiguous), D row-major FP32.  N % 16 == 0, 16 <= N <= 256, K % 64 == 0.
__global__ void __launch_bounds__(kTcThreads)
k_tc_gemm_bf16(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B, float* __restrict__ D,
               int N, int K, int* __restrict__ err) {
    __shared__ __align__(1024) uint8_t sA[128 * kKChunk * 2];
    __shared__ __align__(1024) uint8_t sB[256 * kKChunk * 2];
    __shared__ __align__(8) uint64_t bar, drain;
    __shared__ uint32_t s_taddr;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long m0 = (long long)blockIdx.x * 128;
    const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));

    if (warp == 0) {
        tc::tmem_alloc(&s_taddr, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_init(&drain, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = tc::idesc_bf16_f32(128, N);
    uint32_t phase = 0;
    bool ok = true;

    for (int kc = 0; kc < K && ok; kc += kKChunk) {
        // stage A (128 x 64) and B (N x 64) as K-major core matrices, 16 bytes per copy
        for (int i = tid; i < 128 * (kKChunk / 8); i += kTcThreads) {
            const int row = i / (kKChunk / 8), kb = i % (kKChunk / 8);
            const uint4 v = *reinterpret_cast<const uint4*>(A + (m0 + row) * K + kc + kb * 8);
            *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, kb * 8, kKChunk)) = v;
        }
        for (int i = tid; i < N * (kKChunk / 8); i += kTcThreads) {
            const int row = i / (kKChunk / 8), kb = i % (kKChunk / 8);
            const uint4 v = *reinterpret_cast<const uint4*>(B + (long long)row * K + kc + kb * 8);
            *reinterpret_cast<uint4*>(sB + tc::kmajor_offset(row, kb * 8, kKChunk)) = v;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
            const uint32_t sbo = 128 * (kKChunk / 8);
#pragma unroll
            for (int s = 0; s < kKChunk / 16; ++s) {
                const uint64_t da = tc::smem_desc(a0 + s * 256, 128, sbo);
                const uint64_t db = tc::smem_desc(b0 + s * 256, 128, sbo);
                tc::mma_bf16(taddr, da, db, idesc, (kc > 0 || s > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar);
        }
        // every thread waits: the staging buffers are rewritten next round; a wait that gives
        // up in any thread stops the whole block (the loop's barriers stay matched)
        if (!tc::mbar_wait(&bar, phase, kWaitPolls)) ok = false;
        phase ^= 1;
        ok = __syncthreads_and(ok);
    }
    if (!ok && tid == 0) atomicExch(err, 1);

    if (ok) {
        tc::fence_after_sync();
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const long long row = m0 + warp * 32 + (tid & 31);
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + lane_base + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) D[row * N + c + j] = v[j];
        }
    }
    // also after a wait that gave up: every MMA the issuing thread committed has completed
    // (bounded wait) before the tensor memory is released and the block exits
    if (tid == 0) {
        tc::mma_commit(&drain);
        if (!tc::mbar_wait(&drain, 0, kWaitPolls)) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

// ---------------------------------------------------------------------------
// GELU in its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), with the
// hardware tanh approximation (tanh.approx.f32, relative error ~2^-11, below the
// BF16 rounding of every activation).
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kGeluK0 = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluK1 = 0.044715f;
__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.0f + tanh_fast(kGeluK0 * (x + kGeluK1 * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float t = tanh_fast(kGeluK0 * (z + kGeluK1 * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluK0 * (1.0f + 3.0f * kGeluK1 * z * z);
}

constexpr int align1k(int b) { return (b + 1023) & ~1023; }

// ---------------------------------------------------------------------------
// 3x3 convolution with periodic padding as an implicit GEMM on tcgen05.
//
// Work unit: image b, a segment of 128 pixels of the row, R consecutive rows,
// walked by persistent warp-specialised CTAs.  A row segment is the M = 128
// side of the MMAs; K runs over the input channels of one tap.
//
// Input rows ("halo rows": the segment and one pixel either side, wrapped
// periodically) live in a ring of kRing shared-memory slots, stored channel-
// granule-major: for each group of 8 channels the 130 pixels' 16 bytes are
// contiguous.  Consecutive pixels are then 16 bytes apart, so the A operand of
// a tap with column shift dx - 128 consecutive pixels starting at pixel 1 + dx -
// is a plain descriptor offset (leading byte offset 130 * 16 between channel
// granules, stride byte offset 128 between 8-pixel groups).
//
// Output rows are computed in groups of G.  Output row j reads halo rows j,
// j + 1, j + 2 (taps dy = -1, 0, +1), so one halo row i feeds up to three
// output rows of a group, each through its own tap: the weights are stored
// per column shift dx as three consecutive blocks [dy = +1; dy = 0; dy = -1]
// of COUT x CIN, and one MMA with N = COUT x (number of output rows fed)
// multiplies halo row i by the consecutive blocks of those rows into their
// consecutive accumulator columns.  For COUT = 64 that is mostly N = 192, at
// the tensor core's full rate, against N = 64 for one row at a time (measured:
// 48 cycles per 128 x 64 x 16 MMA, 64 per 128 x 128 x 16).  The accumulator of
// a group (G COUT columns) is zeroed by the epilogue after reading, so every
// MMA accumulates.
//
// Roles, connected by mbarriers (every wait bounded, plus a shared abort flag):
//   producer warps  fill halo rows with cp.async, up to kMaxPending rows in
//                   flight; full[slot] when a row has landed, empty[slot]
//                   when its last MMA has completed
//   MMA warp        one thread issues, per halo row of a group, the MMAs of
//                   the 3 column shifts x CIN / 16 channel slices, then commits
//                   acc_full[a] at the end of the group
//   epilogue warps  per output row of a finished group (warp w: TMEM lanes
//                   32 (w % 4).., half w / 4 of the COUT columns): bias, GELU
//                   (when ACT), Y (and the pre-activation Z when asked),
//                   staged through shared memory (16-byte chunks XOR-swizzled
//                   by pixel) and written as contiguous runs; then the group's
//                   columns are zeroed and the accumulator released
constexpr int kEpiWarps = 8;
constexpr int kProdWarps = 3;
constexpr int kMmaWarp = kEpiWarps;
constexpr int kConvThreads = 32 * (kEpiWarps + 1 + kProdWarps);
constexpr int kHaloPix = 130;
constexpr int kRing = 6;
constexpr int kMaxPending = 3;      // halo rows in flight per producer thread (<= kRing - 3)

template <int CIN, int COUT>
struct ConvRows {
    static constexpr int G = COUT >= 64 ? 4 : 8;                // output rows per group
    static constexpr int KT = 9 * CIN;
    static constexpr int GR = CIN / 8;                          // 16-byte channel granules per pixel
    static constexpr int kSlot = GR * kHaloPix * 16;            // bytes of one halo row
    static constexpr int kW = align1k(COUT * KT * 2);           // bytes of the weight blocks
    static constexpr int KC = COUT / 8;                         // 16-byte chunks of one output pixel
    static constexpr int kStage = 32 * COUT * 2;                // bytes of one staged 32-pixel block
    static constexpr int kSmem = kW + kRing * kSlot + 4 * 2 * kStage;
    static constexpr uint32_t kAcc = G * COUT;                  // accumulator columns of a group
    static constexpr uint32_t kTmem = 2 * kAcc;                 // two accumulators
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 64, "tile shape");
    static_assert(kTmem <= 512 && (kTmem & (kTmem - 1)) == 0, "tensor memory");
    static_assert(3 * COUT <= 256, "MMA N");
    static_assert((KC & (KC - 1)) == 0, "chunk swizzle needs a power of two");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

// Bounded wait that also gives up once another role has raised `abort`.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
    for (long long i = 0; i < kWaitPolls; i += 256) {
        if (tc::mbar_wait(bar, parity, 256)) return true;
        if (*abort) return false;
    }
    return false;
}
__device__ __forceinline__ void raise_abort(volatile int* abort, int* err) {
    *abort = 1;
    atomicExch(err, 1);
}

// The work unit sequence every role walks.  A unit of `rows` output rows has
// ceil(rows / G) groups and reads ceil(rows / G) G + 2 halo rows (rows past
// the unit wrap periodically; their outputs are discarded).
struct ConvUnits {
    int H, Wd, R, G, nseg, nchunk;
    long long n;
    __device__ ConvUnits(int B, int H_, int W_, int R_, int G_) : H(H_), Wd(W_), R(R_), G(G_) {
        nseg = (Wd + 127) / 128;
        nchunk = (H + R - 1) / R;
        n = (long long)B * nseg * nchunk;
    }
    __device__ void decode(long long unit, int& b, int& y0, int& rows, int& x0) const {
        const int seg = (int)(unit % nseg);
        const long long t = unit / nseg;
        const int chunk = (int)(t % nchunk);
        b = (int)(t / nchunk);
        y0 = chunk * R;
        rows = min(R, H - y0);
        x0 = seg * 128;
    }
    __device__ int groups(int rows) const { return (rows + G - 1) / G; }
    __device__ int halos(int rows) const { return groups(rows) * G + 2; }
};

template <int CIN, int COUT, bool ACT, bool STORE_Z>
__global__ void __launch_bounds__(kConvThreads, 1)
k_conv3x3(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias,
          __nv_bfloat16* __restrict__ Y, __nv_bfloat16* __restrict__ Z, int B, int H, int Wd, int R,
          int* __restrict__ err) {
    using Cfg = ConvRows<CIN, COUT>;
    constexpr int G = Cfg::G;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kRing], empty[kRing], acc_full[2], acc_empty[2], mma_done;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    volatile int* abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(&s_taddr, Cfg::kTmem);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < kRing; ++i) {
            tc::mbar_init(&full[i], 32 * kProdWarps);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], 32 * kEpiWarps);
        }
        tc::mbar_init(&mma_done, 1);
    }
    // weight blocks: block ((dx + 1) * 3 + (1 - dy)) holds W[.][tap (dy, dx)][.] as COUT x CIN,
    // K-major core matrices over the stacked 9 COUT rows (stride byte offset 16 CIN)
    const uint32_t w0 = tc::smem_addr(smem), ring0 = w0 + Cfg::kW;
    for (int i = tid; i < 9 * COUT * (CIN / 8); i += kConvThreads) {
        const int row = i / (CIN / 8), kb = i - row * (CIN / 8);
        const int blk = row / COUT, co = row - blk * COUT;
        const int dxi = blk / 3, dy = 1 - (blk - dxi * 3);
        const int tap = 3 * (dy + 1) + dxi;
        tc::cp_async16(w0 + tc::kmajor_offset(row, kb * 8, CIN), Wt + ((long long)co * 9 + tap) * CIN + kb * 8);
    }
    tc::cp_async_commit();
    __syncthreads();                    // barrier inits and s_taddr visible
    const uint32_t taddr = s_taddr;
    if (warp < kEpiWarps) {             // both accumulators start at zero
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        for (uint32_t c = (uint32_t)(warp >> 2) * 32; c < Cfg::kTmem; c += 64) {
            if constexpr (Cfg::kTmem >= 64) tc::tmem_zero32(taddr + lanes + c);
        }
    }
    tc::cp_async_wait<0>();
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const ConvUnits U(B, H, Wd, R, G);

    if (warp > kMmaWarp) {
        // ---------------- producers ----------------
        // Halo rows are issued in stream order h = 0, 1, ...; a row is announced
        // (full[slot]) as soon as this thread's copies of it have landed, also
        // while the producer waits for a free slot, so that announcing never
        // depends on the consumer releasing a later slot.
        const int pt = tid - 32 * (kMmaWarp + 1);
        constexpr int np = 32 * kProdWarps;
        uint32_t h = 0, announced = 0;
        bool ok = true;
        auto announce_oldest = [&]() {
            tc::cp_async_wait_dyn((int)(h - announced) - 1);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&full[announced % kRing]);
            ++announced;
        };
        for (long long unit = blockIdx.x; unit < U.n && ok; unit += gridDim.x) {
            int b, y0, rows, x0;
            U.decode(unit, b, y0, rows, x0);
            const __nv_bfloat16* Xb = X + (long long)b * H * Wd * CIN;
            const int nh = U.halos(rows);
            for (int i = 0; i < nh; ++i, ++h) {
                const uint32_t slot = h % kRing, par = ((h / kRing) & 1u) ^ 1u;
                while (announced < h && (h - announced >= (uint32_t)kMaxPending || !tc::mbar_test(&empty[slot], par)))
                    announce_oldest();
                if (!wait_or_abort(&empty[slot], par, abort)) {
                    raise_abort(abort, err);
                    ok = false;
                    break;
                }
                int yi = (y0 - 1 + i) % H;
                yi = yi < 0 ? yi + H : yi;
                const __nv_bfloat16* src = Xb + (long long)yi * Wd * CIN;
                const uint32_t dst = ring0 + slot * Cfg::kSlot;
                for (int idx = pt; idx < kHaloPix * Cfg::GR; idx += np) {
                    const int pix = idx / Cfg::GR, g = idx - pix * Cfg::GR;
                    int x = x0 - 1 + pix;
                    x = x < 0 ? x + Wd : (x >= Wd ? x % Wd : x);
                    tc::cp_async16(dst + (uint32_t)(g * (kHaloPix * 16) + pix * 16),
                                   src + (long long)x * CIN + g * 8);
                }
                tc::cp_async_commit();
            }
        }
        while (announced < h) announce_oldest();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t idesc[3];
#pragma unroll
            for (int n = 0; n < 3; ++n) idesc[n] = tc::idesc_bf16_f32(128, COUT * (n + 1));
            uint32_t hb = 0, gc = 0;
            bool ok = true;
            for (long long unit = blockIdx.x; unit < U.n && ok; unit += gridDim.x) {
                int b, y0, rows, x0;
                U.decode(unit, b, y0, rows, x0);
                const int ng = U.groups(rows);
                int waited = 0;                       // halo rows of this unit already waited for
                for (int g = 0; g < ng && ok; ++g, ++gc) {
                    const uint32_t a = gc & 1u, u = gc >> 1;
                    ok = wait_or_abort(&acc_empty[a], (u & 1u) ^ 1u, abort);
                    const int j0 = g * G;
                    for (int i = j0; i < j0 + G + 2 && ok; ++i) {
                        const uint32_t hh = hb + (uint32_t)i, slot = hh % kRing;
                        if (i >= waited) {
                            ok = wait_or_abort(&full[slot], (hh / kRing) & 1u, abort);
                            waited = i + 1;
                            tc::fence_proxy_async_smem();
                        }
                        if (!ok) break;
                        tc::fence_after_sync();
                        // output rows jlo..jhi of the group read halo row i, through blocks b0.. of each dx
                        const int jlo = max(j0, i - 2), jhi = min(j0 + G - 1, i);
                        const int nr = jhi - jlo + 1, b0 = jlo - i + 2;
                        const uint32_t id = nr == 1 ? idesc[0] : (nr == 2 ? idesc[1] : idesc[2]);
                        const uint32_t dcol = taddr + a * Cfg::kAcc + (uint32_t)(COUT * (jlo - j0));
                        const uint32_t arow = ring0 + slot * Cfg::kSlot;
#pragma unroll
                        for (int dxi = 0; dxi < 3; ++dxi) {
                            const uint32_t brow = w0 + (uint32_t)(((dxi * 3 + b0) * COUT / 8) * (CIN * 16));
#pragma unroll
                            for (int sk = 0; sk < CIN / 16; ++sk) {
                                const uint64_t da = tc::smem_desc(arow + (uint32_t)(dxi * 16 + 2 * sk * kHaloPix * 16),
                                                                  kHaloPix * 16, 128);
                                const uint64_t db = tc::smem_desc(brow + (uint32_t)(256 * sk), 128, CIN * 16);
                                tc::mma_bf16(dcol, da, db, id, 1u);
                            }
                        }
                        // halo row i is released by the group of output row i (the unit's last group
                        // for the rows past it)
                        if (min(i / G, ng - 1) == g) tc::mma_commit(&empty[slot]);
                    }
                    if (ok) tc::mma_commit(&acc_full[a]);
                }
                hb += (uint32_t)U.halos(rows);
            }
            if (!ok) raise_abort(abort, err);
            // every MMA this thread issued has completed before TMEM is released
            tc::mma_commit(&mma_done);
            if (!tc::mbar_wait(&mma_done, 0, kWaitPolls)) raise_abort(abort, err);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        constexpr int CH = COUT / 2, KC = Cfg::KC;
        const int q = warp & 3, half = warp >> 2, pt = half * 32 + lane;
        uint8_t* stage = smem + Cfg::kW + kRing * Cfg::kSlot + q * 2 * Cfg::kStage;
        int sbuf = 0;
        // stage this thread's CH values (packed BF16) of pixel `lane`, then copy the pair's
        // 32 pixels to dst (pixel 0 of the block) as 16-byte chunks, nvalid pixels
        auto emit = [&](const uint32_t (&pk)[CH / 2], __nv_bfloat16* dst, int nvalid) {
            uint8_t* st = stage + sbuf * Cfg::kStage;
#pragma unroll
            for (int c0 = 0; c0 < CH; c0 += 8) {
                const int k = (half * CH + c0) / 8;
                *reinterpret_cast<uint4*>(st + lane * (KC * 16) + ((k ^ (lane & (KC - 1))) * 16)) =
                    make_uint4(pk[c0 / 2], pk[c0 / 2 + 1], pk[c0 / 2 + 2], pk[c0 / 2 + 3]);
            }
            asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");
            for (int idx = pt; idx < 32 * KC; idx += 64) {
                const int p = idx / KC, k = idx - p * KC;
                if (p < nvalid)
                    *reinterpret_cast<uint4*>(dst + (long long)p * COUT + k * 8) =
                        *reinterpret_cast<const uint4*>(st + p * (KC * 16) + ((k ^ (p & (KC - 1))) * 16));
            }
            sbuf ^= 1;
        };
        float breg[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) breg[c] = bias[half * CH + c];
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        // After a failure the warp keeps walking its rows without waiting or storing, so
        // that the pair's named barriers stay matched.
        uint32_t gc = 0;
        bool ok = true;
        for (long long unit = blockIdx.x; unit < U.n; unit += gridDim.x) {
            int b, y0, rows, x0;
            U.decode(unit, b, y0, rows, x0);
            const int ng = U.groups(rows);
            for (int g = 0; g < ng; ++g, ++gc) {
                const uint32_t a = gc & 1u, u = gc >> 1;
                if (ok && !wait_or_abort(&acc_full[a], u & 1u, abort)) {
                    raise_abort(abort, err);
                    ok = false;
                }
                if (ok) tc::fence_after_sync();
                const int nvalid = ok ? min(32, Wd - (x0 + q * 32)) : 0;
                for (int k = 0; k < G && g * G + k < rows; ++k) {
                    float v[CH];
                    if (ok) {
                        const uint32_t tb = taddr + lanes + a * Cfg::kAcc + (uint32_t)(k * COUT + half * CH);
                        if constexpr (CH == 32) {
                            tc::tmem_ld32(tb, v);
                        } else {
                            static_assert(CH == 8, "column split");
                            tc::tmem_ld8(tb, v);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < CH; ++c) v[c] = 0.0f;
                    }
                    const long long pix0 = ((long long)b * H + y0 + g * G + k) * Wd + x0 + q * 32;
                    uint32_t pz[CH / 2], py[CH / 2];
#pragma unroll
                    for (int c = 0; c < CH; c += 2) {
                        const float z0 = v[c] + breg[c], z1 = v[c + 1] + breg[c + 1];
                        const __nv_bfloat162 zz = __floats2bfloat162_rn(z0, z1);
                        pz[c / 2] = *reinterpret_cast<const uint32_t*>(&zz);
                        const __nv_bfloat162 yy = ACT ? __floats2bfloat162_rn(gelu(z0), gelu(z1)) : zz;
                        py[c / 2] = *reinterpret_cast<const uint32_t*>(&yy);
                    }
                    emit(py, Y + pix0 * COUT, nvalid);
                    if (STORE_Z) emit(pz, Z + pix0 * COUT, nvalid);
                }
                if (ok) {
                    // zero the group's columns of these lanes for the next use, then release
                    for (uint32_t c = (uint32_t)half * 32; c < Cfg::kAcc; c += 64) tc::tmem_zero32(taddr + lanes + a * Cfg::kAcc + c);
                    tc::fence_before_sync();
                    tc::mbar_arrive(&acc_empty[a]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, Cfg::kTmem);
    }
}

template <int CIN, int COUT, bool ACT, bool STORE_Z>
int launch_conv(const void* X, const void* W, const float* bias, void* Y, void* Z, long long B, long long H,
                long long Wd, int* err, cudaStream_t s) {
    using Cfg = ConvRows<CIN, COUT>;
    static int slots = 0;                    // resident CTAs on the device
    if (!slots) {
        auto fn = k_conv3x3<CIN, COUT, ACT, STORE_Z>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem) != cudaSuccess)
            return VLBM_ECUDA;
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kConvThreads, Cfg::kSmem) != cudaSuccess)
            return VLBM_ECUDA;
        // resident CTAs per SM: their accumulators must fit the 512 TMEM columns
        per_sm = std::max(1, std::min(per_sm, (int)(512 / Cfg::kTmem)));
        slots = sms * per_sm;
    }
    // rows per unit (a multiple of the group size): fewest waves of units, counting the
    // two halo rows of each unit
    const long long nseg = (Wd + 127) / 128;
    constexpr int G = Cfg::G;
    int R = G;
    double best = 1e300;
    for (int r : {8 * G, 4 * G, 2 * G, G}) {
        const long long units = B * nseg * ((H + r - 1) / r);
        const double cost = (double)((units + slots - 1) / slots) * (r + 2);
        if (cost < best - 1e-9) {
            best = cost;
            R = r;
        }
    }
    const long long units = B * nseg * ((H + R - 1) / R);
    const unsigned grid = (unsigned)std::min<long long>(units, slots);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_conv3x3<CIN, COUT, ACT, STORE_Z><<<grid, kConvThreads, Cfg::kSmem, s>>>(
        (const __nv_bfloat16*)X, (const __nv_bfloat16*)W, bias, (__nv_bfloat16*)Y, (__nv_bfloat16*)Z, (int)B, (int)H,
        (int)Wd, R, err);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

template <int CIN, int COUT>
int launch_conv_act(const void* X, const void* W, const float* bias, void* Y, void* Z, long long B, long long H,
                    long long Wd, int act, int* err, cudaStream_t s) {
    if (act && Z) return launch_conv<CIN, COUT, true, true>(X, W, bias, Y, Z, B, H, Wd, err, s);
    if (act) return launch_conv<CIN, COUT, true, false>(X, W, bias, Y, nullptr, B, H, Wd, err, s);
    return launch_conv<CIN, COUT, false, false>(X, W, bias, Y, nullptr, B, H, Wd, err, s);
}

// ---------------------------------------------------------------------------
// Weight and bias gradients of a periodic 3x3 convolution, on tcgen05:
//   G[co][tap * CIN + ci] += sum_p X[p + tap][ci] dZ[p][co],   Gb[co] += sum_p dZ[p][co]
// as a GEMM with M = rows (tap, ci) plus one row of ones (which yields the bias
// gradient), N = COUT and K = pixels.  Both operands are MN-major: NHWC memory
// holds the channels of a pixel contiguously, so each 16-byte granule (8
// channels of one pixel) is copied unchanged by cp.async to its place, with no
// transposition.  A stage holds KP pixels:
//   A: 128-byte swizzled MN-major atoms of 64 rows (tap, ci) x KP pixels, one
//      128-byte row per pixel: the 8 granules one pixel contributes to an atom
//      land in 8 different bank groups.  Rows from KT on are constant: the row of
//      ones, then zeros up to whole 128-row tiles;
//   B: the same for dZ when COUT is a multiple of 64, else no-swizzle MN-major
//      [output channel group][pixel][16 B].
// Each CTA accumulates all 128-row tiles of M in tensor memory (TILES x COUT
// columns) over a contiguous range of pixels (split K) and adds its partial
// sums to G / Gb with FP32 atomics.  Roles, connected by mbarriers (every wait
// bounded, plus a shared abort flag): 8 producer warps fill STAGES stages with
// cp.async, up to kWgradPending chunks in flight per thread (full[stage] once a
// chunk has landed); one thread issues the chunk's TILES x KP / 16 MMAs and
// releases the stage (empty[stage]); at the end the producer warps read the
// accumulators.
constexpr int kWgradPending = 3;    // chunks in flight per producer thread (cp.async groups waited on: <= 3)

template <int CIN, int COUT>
struct WgradCfg {
    static constexpr int PRODUCERS = 256;                 // 8 warps copy (and add the sums at the end)
    static constexpr int THREADS = PRODUCERS + 32;        // + 1 warp whose first thread issues the MMAs
    static constexpr int KP = 32;                         // pixels per stage: two K = 16 MMA steps
    static constexpr int KT = 9 * CIN;                    // rows (tap, ci); row KT is the row of ones
    static constexpr int TILES = (KT + 1 + 127) / 128;
    static constexpr int CG = CIN / 8, BG = COUT / 8;     // 16-byte channel groups of X and dZ
    static constexpr int ATOM = KP * 128;                  // one swizzled atom of 64 rows over the stage's pixels
    static constexpr int GROUP = KP * 16;                 // no-swizzle B: one 8-channel group over the pixels
    static constexpr bool B_SW = COUT % 64 == 0;
    static constexpr int A_BYTES = TILES * 2 * ATOM;
    static constexpr int B_BYTES = B_SW ? COUT / 64 * ATOM : BG * GROUP;
    static constexpr int CONST_ATOM = KT / 64;            // first atom holding constant rows
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = 225 * 1024 / STAGE < 5 ? 225 * 1024 / STAGE : 5;
    static constexpr int SMEM = STAGES * STAGE + 1024;    // + slack for 1024-byte alignment
    static constexpr int COLS = TILES * COUT;
    static constexpr uint32_t NCOL = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static constexpr int TSTEP = PRODUCERS / (KP * CG);   // taps one pass of the producers covers
    static_assert(CIN % 8 == 0 && COUT % 16 == 0 && COUT <= 256, "operand shapes");
    static_assert(PRODUCERS % (KP * CG) == 0 && KP * BG <= PRODUCERS, "one granule per thread and pass");
    static_assert(COLS <= 512 && STAGES > kWgradPending, "tensor memory / shared memory budget");
    static_assert(KT % 8 == 0 && STAGE % 1024 == 0 && KP % 16 == 0, "atom alignment");
};

// Byte offset of granule (8 rows starting at row r0, pixel p) in a stage's swizzled operand.
template <int KP>
__device__ __forceinline__ uint32_t sw128_granule(int r0, int p) {
    return (uint32_t)((r0 >> 6) * (KP * 128) + p * 128 + ((((r0 >> 3) & 7) ^ (p & 7)) << 4));
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(WgradCfg<CIN, COUT>::THREADS, 1)
k_conv3x3_wgrad(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ dZ, float* __restrict__ G,
                float* __restrict__ Gb, int B, int H, int Wd, int chunks_per_cta, int* __restrict__ err) {
    using C = WgradCfg<CIN, COUT>;
    constexpr int S = C::STAGES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // swizzle atoms need 1024-byte aligned shared addresses
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    volatile int* abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int npix = B * H * Wd;
    const int nchunks = (npix + C::KP - 1) / C::KP;
    const int c_begin = blockIdx.x * chunks_per_cta;
    const int n = max(0, min(c_begin + chunks_per_cta, nchunks) - c_begin);
    if (warp == 0) {
        tc::tmem_alloc(&s_taddr, C::NCOL);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], C::PRODUCERS);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&done, 1);
        s_abort = 0;
    }
    // constant rows of every stage: row KT is 1.0 (first element of its granule), later rows zero
    constexpr int kConstGroups = (C::TILES * 128 - C::CONST_ATOM * 64) / 8;
    for (int i = tid; i < S * kConstGroups * C::KP; i += C::THREADS) {
        const int s = i / (kConstGroups * C::KP), j = i - s * (kConstGroups * C::KP);
        const int r0 = C::CONST_ATOM * 64 + 8 * (j / C::KP), p = j % C::KP;
        if (r0 >= C::KT)
            *reinterpret_cast<uint4*>(smem + s * C::STAGE + sw128_granule<C::KP>(r0, p)) =
                make_uint4(r0 == C::KT ? 0x00003F80u : 0u, 0u, 0u, 0u);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const uint32_t sbase = tc::smem_addr(smem);

    if (warp < C::PRODUCERS / 32) {
        // ---------------- producers ----------------
        // this thread's granules: pixel pa, channel group ga of taps ta0, ta0 + TSTEP, ...; dZ pixel pb, group gb.
        // A chunk is announced (full[stage]) once this thread's copies of it have landed, also while the
        // thread waits for a free stage, so that announcing never depends on a later stage being released.
        const int pa = (tid % (C::KP * C::CG)) / C::CG, ga = tid % C::CG, ta0 = tid / (C::KP * C::CG);
        const bool b_thread = tid < C::KP * C::BG;
        const int pb = tid / C::BG, gb = tid % C::BG;
        const uint32_t b_off = C::A_BYTES + (C::B_SW ? sw128_granule<C::KP>(8 * gb, pb) : (uint32_t)(gb * C::GROUP + pb * 16));
        int qa = c_begin * C::KP + pa, qb = c_begin * C::KP + pb;
        int x = 0, y = 0, b = 0;                          // coordinates of pixel qa, advanced by KP per chunk
        if (qa < npix) {
            x = qa % Wd;
            const int t = qa / Wd;
            y = t % H;
            b = t / H;
        }
        int issued = 0, announced = 0;
        auto announce_oldest = [&]() {
            tc::cp_async_wait_dyn(issued - announced - 1);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&full[announced % S]);
            ++announced;
        };
        for (int c = 0; c < n; ++c) {
            const int s = c % S;
            const uint32_t par = ((c / S) & 1) ^ 1;
            while (announced < issued && (issued - announced >= kWgradPending || !tc::mbar_test(&empty[s], par)))
                announce_oldest();
            if (!wait_or_abort(&empty[s], par, abort)) {
                raise_abort(abort, err);
                break;
            }
            const uint32_t sa = sbase + s * C::STAGE;
            const bool valid = qa < npix;
            const int ys[3] = {y == 0 ? H - 1 : y - 1, y, y == H - 1 ? 0 : y + 1};
            const int xs[3] = {x == 0 ? Wd - 1 : x - 1, x, x == Wd - 1 ? 0 : x + 1};
#pragma unroll
            for (int i = 0; i < (9 + C::TSTEP - 1) / C::TSTEP; ++i) {
                const int tap = ta0 + i * C::TSTEP;
                if (tap < 9) {
                    const __nv_bfloat16* src = X + ((long long)(b * H + ys[tap / 3]) * Wd + xs[tap % 3]) * CIN + ga * 8;
                    tc::cp_async16_ca_zfill(sa + sw128_granule<C::KP>(tap * CIN + 8 * ga, pa), valid ? src : X,
                                            valid ? 16u : 0u);
                }
            }
            if (b_thread) {
                const bool vb = qb < npix;
                tc::cp_async16_ca_zfill(sa + b_off, vb ? dZ + (long long)qb * COUT + gb * 8 : dZ, vb ? 16u : 0u);
            }
            tc::cp_async_commit();
            ++issued;
            qa += C::KP;
            qb += C::KP;
            for (x += C::KP; x >= Wd; x -= Wd)
                if (++y == H) {
                    y = 0;
                    ++b;
                }
        }
        while (announced < issued) announce_oldest();
    } else if ((tid & 31) == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = tc::idesc_bf16_f32_mn(128, COUT);
        bool ok = true;
        for (int c = 0; c < n && ok; ++c) {
            const int s = c % S;
            if (!wait_or_abort(&full[s], (c / S) & 1, abort)) {
                raise_abort(abort, err);
                ok = false;
                break;
            }
            tc::fence_proxy_async_smem();
            tc::fence_after_sync();
            const uint32_t a0 = sbase + s * C::STAGE, b0 = a0 + C::A_BYTES;
#pragma unroll
            for (int t = 0; t < C::TILES; ++t)
#pragma unroll
                for (int k = 0; k < C::KP / 16; ++k) {
                    // 16 pixels = two 8-row groups further along K
                    const uint64_t da = tc::smem_desc_sw128(a0 + t * 2 * C::ATOM + k * 2048, C::ATOM, 1024);
                    const uint64_t db = C::B_SW ? tc::smem_desc_sw128(b0 + k * 2048, C::ATOM, 1024)
                                                : tc::smem_desc(b0 + k * 256, 128, C::GROUP);
                    tc::mma_bf16(taddr + (uint32_t)(t * COUT), da, db, idesc, (c > 0 || k > 0) ? 1u : 0u);
                }
            tc::mma_commit(&empty[s]);
        }
        // arrives once every MMA above has completed; the issuer waits for it (bounded) also after
        // an abort, so that no MMA still targets the tensor memory released below
        if (n > 0) {
            tc::mma_commit(&done);
            if (!tc::mbar_wait(&done, 0, kWaitPolls)) raise_abort(abort, err);
        }
    }
    // ---------------- epilogue: the producer warps add the partial sums ----------------
    if (warp < C::PRODUCERS / 32 && n > 0) {
        if (wait_or_abort(&done, 0, abort)) {
            tc::fence_after_sync();
            const int quarter = warp & 3;                // a warp reads TMEM lanes 32 * (warp % 4) ..
            const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
            for (int t = warp >> 2; t < C::TILES; t += C::PRODUCERS / 128) {
                const int r = t * 128 + quarter * 32 + (tid & 31);
#pragma unroll
                for (int c = 0; c < COUT; c += 16) {
                    float v[16];
                    tc::tmem_ld16(taddr + lane_base + (uint32_t)(t * COUT + c), v);
                    if (r < C::KT) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) atomicAdd(G + (long long)(c + j) * C::KT + r, v[j]);
                    } else if (r == C::KT) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) atomicAdd(Gb + c + j, v[j]);
                    }
                }
            }
        } else {
            raise_abort(abort, err);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, C::NCOL);
}

// ---------------------------------------------------------------------------
// Elementwise kernels of the surrogate's training step.

// Per-channel factors passed by value (channels <= 16).
struct ChanScale {
    float v[16];
};

// u [B][C][H][W] FP32 -> X [B][H][W][16] BF16, channel c scaled by in.v[c]; when DIV, channel C
// holds in.v[C] times the periodic central-difference divergence of channels 0, 1 (unit spacing),
// taken in FP32 before the rounding to BF16 (it is ~1e-3 of the velocity, below BF16's resolution
// of the velocity itself).  Remaining channels are zero.
// Training noise: a standard normal draw per (step, pixel, channel) from a counter-based
// generator (the splitmix64 finaliser of Steele, Lea and Flood, applied to the counter),
// turned into a normal deviate by the Box-Muller transform.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float normal_draw(uint64_t key) {
    const uint64_t h1 = mix64(key * 2 + 1), h2 = mix64(key * 2 + 2);
    const float u1 = ((float)(h1 >> 40) + 1.0f) * (1.0f / 16777216.0f);      // (0, 1]
    const float u2 = (float)(h2 >> 40) * (1.0f / 16777216.0f);               // [0, 1)
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

template <bool DIV>
__global__ void k_pack_input(const float* __restrict__ u, __nv_bfloat16* __restrict__ X, int H, int W, long long npix,
                             int C, ChanScale in, const ChanScale* noise, uint64_t noise_key) {
    const long long plane = (long long)H * W;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const long long b = p / plane, q = p - b * plane;
    __align__(16) __nv_bfloat16 e[16];
#pragma unroll
    for (int c = 0; c < 16; ++c)
        e[c] = __float2bfloat16_rn(c < C ? u[(b * C + c) * plane + q] * in.v[c] : 0.0f);
    if (DIV) {
        const int x = (int)(q % W), y = (int)(q / W);
        const int xp = x + 1 == W ? 0 : x + 1, xm = x == 0 ? W - 1 : x - 1;
        const int yp = y + 1 == H ? 0 : y + 1, ym = y == 0 ? H - 1 : y - 1;
        const float* ux = u + b * C * plane;
        const float* uy = ux + plane;
        const float d = 0.5f * (ux[(long long)y * W + xp] - ux[(long long)y * W + xm]) +
                        0.5f * (uy[(long long)yp * W + x] - uy[(long long)ym * W + x]);
        e[C] = __float2bfloat16_rn(d * in.v[C]);
    }
    if (noise) {
        const int n_in = C + (DIV ? 1 : 0);
        for (int c = 0; c < n_in; ++c) {
            const float sg = noise->v[c];
            if (sg != 0.0f) {
                const float x = __bfloat162float(e[c]) + sg * normal_draw(noise_key + (uint64_t)(p * 16 + c));
                e[c] = __float2bfloat16_rn(x);
            }
        }
    }
    reinterpret_cast<uint4*>(X + p * 16)[0] = reinterpret_cast<const uint4*>(e)[0];
    reinterpret_cast<uint4*>(X + p * 16)[1] = reinterpret_cast<const uint4*>(e)[1];
}

// Y [B][H][W][16] BF16 (channels 0 .. C-1) -> out [B][C][H][W] FP32 = base + sc.v[c] Y
// (base may be NULL: out = sc.v[c] Y).  out may alias base.
__global__ void k_unpack_output(const __nv_bfloat16* __restrict__ Y, const float* base, float* out, ChanScale sc,
                                long long plane, long long npix, int C) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const long long b = p / plane, q = p - b * plane;
    for (int c = 0; c < C; ++c) {
        const long long i = (b * C + c) * plane + q;
        const float y = sc.v[c] * __bfloat162float(Y[p * 16 + c]);
        out[i] = base ? base[i] + y : y;
    }
}

// Curl output (VLBM_SUR_FEATURE_CURL): channel 0 of Y is a stream function psi and the
// velocity increment is (D_y psi, -D_x psi) with periodic central differences
// D_y psi = (psi(y+1) - psi(y-1)) / 2, which the same differences see as divergence-free.
// out = base + sc.v[0] (D_y psi, -D_x psi) for channels 0, 1 and base + sc.v[c] Y[c] for c >= 2.
__device__ __forceinline__ float psi_at(const __nv_bfloat16* Y, long long img, int y, int x, int W) {
    return __bfloat162float(Y[(img + (long long)y * W + x) * 16]);
}
__global__ void k_unpack_curl(const __nv_bfloat16* __restrict__ Y, const float* base, float* out, ChanScale sc,
                              int H, int W, long long npix, int C) {
    const long long plane = (long long)H * W;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const long long b = p / plane, q = p - b * plane, img = b * plane;
    const int x = (int)(q % W), y = (int)(q / W);
    const int xp = x + 1 == W ? 0 : x + 1, xm = x == 0 ? W - 1 : x - 1;
    const int yp = y + 1 == H ? 0 : y + 1, ym = y == 0 ? H - 1 : y - 1;
    const float dy = 0.5f * (psi_at(Y, img, yp, x, W) - psi_at(Y, img, ym, x, W));
    const float dx = 0.5f * (psi_at(Y, img, y, xp, W) - psi_at(Y, img, y, xm, W));
    const float inc[2] = {sc.v[0] * dy, -sc.v[0] * dx};
    for (int c = 0; c < C; ++c) {
        const long long i = (b * C + c) * plane + q;
        const float d = c < 2 ? inc[c] : sc.v[c] * __bfloat162float(Y[p * 16 + c]);
        out[i] = base ? base[i] + d : d;
    }
}

// Curl-output loss, first pass: residuals r = prediction - target of the two velocity
// channels (FP32, r[p][2]) and of channels c >= 2 (kept in r2 [p][14]); sum of squares into sse.
__global__ void k_curl_residual(const __nv_bfloat16* __restrict__ Y, const float* __restrict__ t,
                                float* __restrict__ r, double* __restrict__ sse, int H, int W, long long npix, int C) {
    const long long plane = (long long)H * W;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float local = 0.0f;
    if (p < npix) {
        const long long b = p / plane, q = p - b * plane, img = b * plane;
        const int x = (int)(q % W), y = (int)(q / W);
        const int xp = x + 1 == W ? 0 : x + 1, xm = x == 0 ? W - 1 : x - 1;
        const int yp = y + 1 == H ? 0 : y + 1, ym = y == 0 ? H - 1 : y - 1;
        const float dy = 0.5f * (psi_at(Y, img, yp, x, W) - psi_at(Y, img, ym, x, W));
        const float dx = 0.5f * (psi_at(Y, img, y, xp, W) - psi_at(Y, img, y, xm, W));
        const float rx = dy - t[(b * C + 0) * plane + q], ry = -dx - t[(b * C + 1) * plane + q];
        r[p * 16 + 0] = rx;
        r[p * 16 + 1] = ry;
        local = rx * rx + ry * ry;
        for (int c = 2; c < C; ++c) {
            const float rc = __bfloat162float(Y[p * 16 + c]) - t[(b * C + c) * plane + q];
            r[p * 16 + c] = rc;
            local += rc * rc;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sse, (double)local);
}

// Curl-output loss, second pass: dY = d(loss)/dY with loss = sum r^2 * inv_count.
// Channel 0 (psi): d(sum r^2)/d psi(p) = r_x(p - y) - r_x(p + y) + r_y(p + x) - r_y(p - x) (the factor 2 of
// the square and the 1/2 of the central difference cancel).
__global__ void k_curl_grad(const float* __restrict__ r, __nv_bfloat16* __restrict__ dY, int H, int W, long long npix,
                            int C, float inv_count) {
    const long long plane = (long long)H * W;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const long long b = p / plane, q = p - b * plane, img = b * plane;
    const int x = (int)(q % W), y = (int)(q / W);
    const int xp = x + 1 == W ? 0 : x + 1, xm = x == 0 ? W - 1 : x - 1;
    const int yp = y + 1 == H ? 0 : y + 1, ym = y == 0 ? H - 1 : y - 1;
    auto at = [&](int yy, int xx, int c) { return r[(img + (long long)yy * W + xx) * 16 + c]; };
    const float g = at(ym, x, 0) - at(yp, x, 0) + at(y, xp, 1) - at(y, xm, 1);
    __align__(16) __nv_bfloat16 e[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) e[c] = __float2bfloat16_rn(0.0f);
    e[0] = __float2bfloat16_rn(g * inv_count);
    for (int c = 2; c < C; ++c) e[c] = __float2bfloat16_rn(2.0f * r[p * 16 + c] * inv_count);
    reinterpret_cast<uint4*>(dY + p * 16)[0] = reinterpret_cast<const uint4*>(e)[0];
    reinterpret_cast<uint4*>(dY + p * 16)[1] = reinterpret_cast<const uint4*>(e)[1];
}

// Average pooling by an integer factor F of fields [B][C][H F][W F] -> [B][C][H][W], FP32;
// the F x F sum is taken in a fixed order (rows, then columns) in FP32.
__global__ void k_pool(const float* __restrict__ in, float* __restrict__ out, long long n_out, int H, int W, int F) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    const int x = (int)(i % W);
    const long long r = i / W;
    const int y = (int)(r % H);
    const long long bc = r / H;
    const long long Wf = (long long)W * F;
    const float* src = in + (bc * H * F + (long long)y * F) * Wf + (long long)x * F;
    float acc = 0.0f;
    for (int dy = 0; dy < F; ++dy)
        for (int dx = 0; dx < F; ++dx) acc += src[dy * Wf + dx];
    out[i] = acc / (float)(F * F);
}

// Training pairs from a snapshot store snaps [n][C][plane]: for entry b,
// u[b] = snaps[idx[b]], target[b][c] = (snaps[idx[b] + 1][c] - snaps[idx[b]][c]) * inv.v[c].
__global__ void k_gather_pairs(const float* __restrict__ snaps, const int64_t* __restrict__ idx, float* __restrict__ u,
                               float* __restrict__ target, long long plane, int C, int batch, ChanScale inv) {
    const long long per_field = plane * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per_field * batch) return;
    const long long b = i / per_field, q = i - b * per_field;
    const long long k = idx[b];
    const float a = snaps[k * per_field + q], c = snaps[(k + 1) * per_field + q];
    u[i] = a;
    target[i] = (c - a) * inv.v[q / plane];
}

// Per-field sums of squares of a - b and of b: out[f][0] += sum (a - b)^2,
// out[f][1] += sum b^2 over the first n values of field f, fields ld values apart
// (FP64 atomics; out zeroed by the caller).
__global__ void k_diff_norms(const float* __restrict__ a, const float* __restrict__ b, double* __restrict__ out,
                             long long n, long long ld) {
    const int f = blockIdx.y;
    const float* pa = a + (long long)f * ld;
    const float* pb = b + (long long)f * ld;
    double d = 0.0, r = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = (double)pa[i] - (double)pb[i], y = pb[i];
        d += x * x;
        r += y * y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, off);
        r += __shfl_xor_sync(0xffffffffu, r, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out + 2 * f, d);
        atomicAdd(out + 2 * f + 1, r);
    }
}

// Per-field statistics of the velocity channels 0, 1 of u [B][C][H][W] (periodic, unit spacing):
//   out[b][0] = sum (u_x^2 + u_y^2) / 2
//   out[b][1] = sum (d_x u_x + d_y u_y)^2            (central differences)
//   out[b][2] = sum |grad u|^2                        (same differences, all four)
// Each thread sums its few pixels' terms in FP32 (one rounding per term, ~6e-8 relative); the
// block reduces the partial sums in FP64 and adds them to out (zeroed by the caller) with one
// atomic per value: FP64 arithmetic per pixel, or an atomic per warp, would leave the kernel
// bound by the GPU's slow FP64 pipe and by contention on the 3 addresses of a state.
__global__ void __launch_bounds__(256)
k_field_stats(const float* __restrict__ u, double* __restrict__ out, int C, int H, int W) {
    const int b = blockIdx.y;
    const long long plane = (long long)H * W;
    const float* ux = u + (long long)b * C * plane;
    const float* uy = ux + plane;
    float ef = 0.0f, df = 0.0f, gf = 0.0f;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < plane; q += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(q % W), y = (int)(q / W);
        const int xp = x + 1 == W ? 0 : x + 1, xm = x == 0 ? W - 1 : x - 1;
        const int yp = y + 1 == H ? 0 : y + 1, ym = y == 0 ? H - 1 : y - 1;
        const long long r = (long long)y * W;
        const float a = ux[q], c = uy[q];
        const float axx = 0.5f * (ux[r + xp] - ux[r + xm]), axy = 0.5f * (ux[(long long)yp * W + x] - ux[(long long)ym * W + x]);
        const float cxx = 0.5f * (uy[r + xp] - uy[r + xm]), cxy = 0.5f * (uy[(long long)yp * W + x] - uy[(long long)ym * W + x]);
        const float dv = axx + cxy;
        ef += 0.5f * (a * a + c * c);
        df += dv * dv;
        gf += (axx * axx + axy * axy) + (cxx * cxx + cxy * cxy);
    }
    double e = ef, d = df, g = gf;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, off);
        d += __shfl_xor_sync(0xffffffffu, d, off);
        g += __shfl_xor_sync(0xffffffffu, g, off);
    }
    __shared__ double red[3][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = e;
        red[1][warp] = d;
        red[2][warp] = g;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[threadIdx.x][w];
        atomicAdd(out + b * 3 + threadIdx.x, t);
    }
}

// The rollout's per-state check, decided on the device so that a checked rollout needs no host round
// trip per step.  From the statistics of the new state (stats) and of the state it was advanced from
// (prev), both [n][3] as k_field_stats writes them:
//   energy step   |E / E_prev - 1| <= step_tol
//   energy drift  |E / E_0 - 1| <= drift_tol
//   divergence    sqrt(D / max(G, 1e-300)) <= r_max[b]
// A state fails when any test fails, NaN included (every comparison with NaN is false; the max
// propagates NaN like numpy's maximum).  mask[b] = 1 for a failing state; counts[b] (b < n) counts
// its failures, counts[n .. n + 2] the failing tests (energy step, energy drift, divergence).
__global__ void k_rollout_check(const double* __restrict__ stats, const double* __restrict__ prev,
                                const double* __restrict__ e0, const double* __restrict__ r_max, int n,
                                double step_tol, double drift_tol, uint8_t* __restrict__ mask,
                                unsigned long long* __restrict__ counts) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double e = stats[3 * b], g = stats[3 * b + 2];
    const double gm = (g != g) ? g : (g > 1e-300 ? g : 1e-300);
    const double r = sqrt(stats[3 * b + 1] / gm);
    const bool b_step = !(fabs(e / prev[3 * b] - 1.0) <= step_tol);
    const bool b_drift = !(fabs(e / e0[b] - 1.0) <= drift_tol);
    const bool b_div = !(r <= r_max[b]);
    const bool bad = b_step || b_drift || b_div;
    mask[b] = bad ? 1 : 0;
    if (bad) counts[b] += 1;
    if (b_step) atomicAdd(counts + n, 1ull);
    if (b_drift) atomicAdd(counts + n + 1, 1ull);
    if (b_div) atomicAdd(counts + n + 2, 1ull);
}

// Mean-squared loss of output channels 0 .. C-1 against t [B][C][H][W]; dY (16 ch) and sum of squares.
__global__ void k_mse_grad(const __nv_bfloat16* __restrict__ Y, const float* __restrict__ t,
                           __nv_bfloat16* __restrict__ dY, double* __restrict__ sse, long long plane, long long npix,
                           float inv_count, int C) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float local = 0.0f;
    if (p < npix) {
        const long long b = p / plane, q = p - b * plane;
        __align__(16) __nv_bfloat16 e[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) e[c] = __float2bfloat16_rn(0.0f);
        for (int c = 0; c < C; ++c) {
            const float d = __bfloat162float(Y[p * 16 + c]) - t[(b * C + c) * plane + q];
            local += d * d;
            e[c] = __float2bfloat16_rn(2.0f * d * inv_count);
        }
        reinterpret_cast<uint4*>(dY + p * 16)[0] = reinterpret_cast<const uint4*>(e)[0];
        reinterpret_cast<uint4*>(dY + p * 16)[1] = reinterpret_cast<const uint4*>(e)[1];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sse, (double)local);
}

// dZ = dY * GELU'(Z), BF16, n elements
__global__ void k_gelu_back(const __nv_bfloat16* __restrict__ dY, const __nv_bfloat16* __restrict__ Z,
                            __nv_bfloat16* __restrict__ dZ, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dZ[i] = __float2bfloat16_rn(__bfloat162float(dY[i]) * gelu_grad(__bfloat162float(Z[i])));
}

// Adam on FP32 master parameters; refreshes the BF16 weights W [cout][9][cin],
// their flipped transpose Wt [cin][9][cout] (tap -> 8 - tap) used for the data
// gradient, and the FP32 bias.  Parameter vector per layer: W then bias.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_refresh_weights(const float* __restrict__ w, __nv_bfloat16* __restrict__ W,
                                  __nv_bfloat16* __restrict__ Wflip, int cin, int cout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = cout * 9 * cin;
    if (i >= n) return;
    const int co = i / (9 * cin), rem = i % (9 * cin), tap = rem / cin, ci = rem % cin;
    const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
    W[i] = h;
    Wflip[((long long)ci * 9 + (8 - tap)) * cout + co] = h;
}

}  // namespace

extern "C" int vlbm_tc_gemm_bf16(const void* A, const void* B, float* D, int64_t M, int64_t N, int64_t K,
                                 int32_t* err_dev, void* stream) {
    if (!A || !B || !D || !err_dev || M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K <= 0 || K % kKChunk)
        return VLBM_EINVAL;
    if (misaligned(A, 16) || misaligned(B, 16)) return VLBM_EINVAL;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_tc_gemm_bf16<<<(unsigned)(M / 128), kTcThreads, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)A, (const __nv_bfloat16*)B, D, (int)N, (int)K, err_dev);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_sur_conv3x3(const void* X, const void* W, const float* bias, void* Y, void* Z, int64_t B,
                                int64_t H, int64_t Wd, int32_t cin, int32_t cout, int32_t act, int32_t* err_dev,
                                void* stream) {
    if (!X || !W || !bias || !Y || !err_dev || B < 1 || H < 1 || Wd < 1) return VLBM_EINVAL;
    // 16-byte copies of X and W and 16-byte stores of Y and Z
    if (misaligned(X, 16) || misaligned(W, 16) || misaligned(Y, 16) || (Z && misaligned(Z, 16))) return VLBM_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    if (cin == 16 && cout == 64) return launch_conv_act<16, 64>(X, W, bias, Y, Z, B, H, Wd, act, err_dev, s);
    if (cin == 64 && cout == 64) return launch_conv_act<64, 64>(X, W, bias, Y, Z, B, H, Wd, act, err_dev, s);
    if (cin == 64 && cout == 16) return launch_conv_act<64, 16>(X, W, bias, Y, Z, B, H, Wd, act, err_dev, s);
    if (cin == 16 && cout == 16) return launch_conv_act<16, 16>(X, W, bias, Y, Z, B, H, Wd, act, err_dev, s);
    return VLBM_EUNSUPPORTED;
}

// ===========================================================================
// The surrogate network: five periodic 3x3 convolutions, 2 -> 64 -> 64 -> 64
// -> 64 -> 2 channels (stored padded to 16 at both ends), GELU after the first
// four, BF16 weights and activations, FP32 accumulation, FP32 master weights
// trained with Adam.  Its input is a velocity field u [B][2][H][W]; its output
// is an increment du of the same shape (the caller scales and adds it).
namespace {

constexpr int kLayers = 5;
constexpr int kCin[kLayers] = {16, 64, 64, 64, 64};
constexpr int kCout[kLayers] = {64, 64, 64, 64, 16};

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int CIN, int COUT>
int launch_wgrad(const void* X, const void* dZ, float* G, float* Gb, long long B, long long H, long long W, int* err,
                 cudaStream_t s) {
    using C = WgradCfg<CIN, COUT>;
    static int slots = 0;
    if (!slots) {
        auto fn = k_conv3x3_wgrad<CIN, COUT>;
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
                cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, C::THREADS, C::SMEM) != cudaSuccess)
            return VLBM_ECUDA;
        // resident CTAs must also fit in the 512 tensor-memory columns of an SM
        per_sm = std::max(1, std::min(per_sm, (int)(512 / C::NCOL)));
        slots = sms * per_sm;
    }
    const long long npix = B * H * W;
    if (npix == 0) return VLBM_OK;
    const long long nchunks = (npix + C::KP - 1) / C::KP;
    const long long per = (nchunks + slots - 1) / slots;      // one wave: contiguous chunk ranges
    const unsigned grid = (unsigned)((nchunks + per - 1) / per);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_conv3x3_wgrad<CIN, COUT><<<grid, C::THREADS, C::SMEM, s>>>((const __nv_bfloat16*)X, (const __nv_bfloat16*)dZ, G,
                                                                  Gb, (int)B, (int)H, (int)W, (int)per, err);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

int conv_any(int cin, int cout, const void* X, const void* W, const float* bias, void* Y, void* Z, long long B,
             long long H, long long Wd, int act, int* err, cudaStream_t s) {
    return vlbm_sur_conv3x3(X, W, bias, Y, Z, B, H, Wd, cin, cout, act, err, s);
}

int wgrad_any(int cin, int cout, const void* X, const void* dZ, float* G, float* Gb, long long B, long long H,
              long long W, int* err, cudaStream_t s) {
    if (cin == 16 && cout == 64) return launch_wgrad<16, 64>(X, dZ, G, Gb, B, H, W, err, s);
    if (cin == 64 && cout == 64) return launch_wgrad<64, 64>(X, dZ, G, Gb, B, H, W, err, s);
    if (cin == 64 && cout == 16) return launch_wgrad<64, 16>(X, dZ, G, Gb, B, H, W, err, s);
    return VLBM_EUNSUPPORTED;
}

}  // namespace

struct vlbm_sur {
    int H = 0, W = 0, C = 2, maxB = 0;
    int features = 0, n_in = 2;
    ChanScale* noise_dev = nullptr;
    bool use_noise = false;
    uint64_t noise_seed = 0, noise_draws = 0;
    ChanScale in_scale{}, out_scale{};
    cudaStream_t stream = nullptr;
    long long off_w[kLayers] = {}, off_b[kLayers] = {}, nparams = 0;
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long adam_t = 0;
    __nv_bfloat16* Wb[kLayers] = {};
    __nv_bfloat16* Wflip[kLayers] = {};
    __nv_bfloat16* X0 = nullptr;
    __nv_bfloat16* Y[kLayers] = {};
    __nv_bfloat16* Z[kLayers - 1] = {};
    __nv_bfloat16* dA = nullptr;
    __nv_bfloat16* dB = nullptr;
    float* zero_bias = nullptr;
    float* resid = nullptr;             // curl-output loss residuals [pixels][16] (curl mode only)
    double* sse = nullptr;
    int* err = nullptr;
};

namespace {

uint64_t mix64_host(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void free_sur(vlbm_sur* s) {
    void* ptrs[] = {s->params, s->grads, s->adam_m, s->adam_v, s->X0,  s->dA,
                    s->dB,     s->zero_bias, s->sse, s->err,    s->noise_dev, s->resid};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < kLayers; ++l) {
        if (s->Wb[l]) cudaFree(s->Wb[l]);
        if (s->Wflip[l]) cudaFree(s->Wflip[l]);
        if (s->Y[l]) cudaFree(s->Y[l]);
        if (l < kLayers - 1 && s->Z[l]) cudaFree(s->Z[l]);
    }
}

int refresh_all(vlbm_sur* s) {
    for (int l = 0; l < kLayers; ++l) {
        const int n = kCout[l] * 9 * kCin[l];
        g_launches.fetch_add(1, std::memory_order_relaxed);
        k_refresh_weights<<<(n + 255) / 256, 256, 0, s->stream>>>(s->params + s->off_w[l], s->Wb[l], s->Wflip[l],
                                                                  kCin[l], kCout[l]);
    }
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

int check_err(vlbm_sur* s) {
    int e = 0;
    if (cudaMemcpyAsync(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return VLBM_ECUDA;
    return e ? VLBM_ETIMEOUT : VLBM_OK;
}

// Forward pass of `batch` fields; keeps the pre-activations (and adds the training
// noise to the inputs, when set) when `train`.
int sur_forward(vlbm_sur* s, const float* u, int batch, bool train) {
    const long long plane = (long long)s->H * s->W, npix = plane * batch;
    const ChanScale* noise = nullptr;
    uint64_t key = 0;
    if (train && s->use_noise) {
        noise = s->noise_dev;
        key = mix64_host(s->noise_seed) + s->noise_draws;
        s->noise_draws += (uint64_t)npix * 16;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (s->features & VLBM_SUR_FEATURE_DIV)
        k_pack_input<true><<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(u, s->X0, s->H, s->W, npix, s->C,
                                                                                  s->in_scale, noise, key);
    else
        k_pack_input<false><<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(u, s->X0, s->H, s->W, npix, s->C,
                                                                                   s->in_scale, noise, key);
    const void* x = s->X0;
    for (int l = 0; l < kLayers; ++l) {
        const bool act = l < kLayers - 1;
        int rc = conv_any(kCin[l], kCout[l], x, s->Wb[l], s->params + s->off_b[l], s->Y[l],
                          (act && train) ? s->Z[l] : nullptr, batch, s->H, s->W, act ? 1 : 0, s->err, s->stream);
        if (rc) return rc;
        x = s->Y[l];
    }
    return VLBM_OK;
}

}  // namespace

extern "C" int vlbm_sur_conv3x3_wgrad(const void* X, const void* dZ, float* G, float* Gb, int64_t B, int64_t H,
                                      int64_t Wd, int32_t cin, int32_t cout, int32_t* err_dev, void* stream) {
    if (!X || !dZ || !G || !Gb || !err_dev || B < 1 || H < 1 || Wd < 1) return VLBM_EINVAL;
    if ((unsigned long long)(B * H * Wd) >= (1ull << 31)) return VLBM_EINVAL;
    if (misaligned(X, 16) || misaligned(dZ, 16)) return VLBM_EINVAL;      // 16-byte cp.async copies
    return wgrad_any(cin, cout, X, dZ, G, Gb, B, H, Wd, err_dev, (cudaStream_t)stream);
}

extern "C" int vlbm_sur_create(int32_t H, int32_t W, int32_t channels, int32_t features, int32_t max_batch,
                               uint64_t seed, void* stream, vlbm_sur** out) {
    if (!out || H < 1 || W < 1 || max_batch < 1 || channels < 1 || channels > 16) return VLBM_EINVAL;
    if (features & ~(VLBM_SUR_FEATURE_DIV | VLBM_SUR_FEATURE_CURL)) return VLBM_EINVAL;
    const int n_in = channels + ((features & VLBM_SUR_FEATURE_DIV) ? 1 : 0);
    if (n_in > 16 || ((features & (VLBM_SUR_FEATURE_DIV | VLBM_SUR_FEATURE_CURL)) && channels < 2))
        return VLBM_EINVAL;
    if ((long long)H * W * max_batch >= (1ll << 31)) return VLBM_EINVAL;
    *out = nullptr;
    vlbm_sur* s = new (std::nothrow) vlbm_sur();
    if (!s) return VLBM_ENOMEM;
    s->H = H;
    s->W = W;
    s->C = channels;
    s->features = features;
    s->n_in = n_in;
    for (int c = 0; c < 16; ++c) s->in_scale.v[c] = s->out_scale.v[c] = 1.0f;
    s->maxB = max_batch;
    s->stream = (cudaStream_t)stream;
    long long off = 0;
    for (int l = 0; l < kLayers; ++l) {
        s->off_w[l] = off;
        off += (long long)kCout[l] * 9 * kCin[l];
        s->off_b[l] = off;
        off += kCout[l];
    }
    s->nparams = off;
    const long long npix = (long long)H * W * max_batch;
    bool okm = true;
    auto alloc = [&](void** p, size_t bytes) {
        if (okm && cudaMalloc(p, bytes) != cudaSuccess) okm = false;
    };
    alloc((void**)&s->params, off * 4);
    alloc((void**)&s->grads, off * 4);
    alloc((void**)&s->adam_m, off * 4);
    alloc((void**)&s->adam_v, off * 4);
    alloc((void**)&s->X0, npix * 16 * 2);
    alloc((void**)&s->dA, npix * 64 * 2);
    alloc((void**)&s->dB, npix * 64 * 2);
    alloc((void**)&s->zero_bias, 64 * 4);
    alloc((void**)&s->sse, sizeof(double));
    alloc((void**)&s->err, sizeof(int));
    alloc((void**)&s->noise_dev, sizeof(ChanScale));
    if (features & VLBM_SUR_FEATURE_CURL) alloc((void**)&s->resid, npix * 16 * sizeof(float));
    for (int l = 0; l < kLayers; ++l) {
        alloc((void**)&s->Wb[l], (size_t)kCout[l] * 9 * kCin[l] * 2);
        alloc((void**)&s->Wflip[l], (size_t)kCout[l] * 9 * kCin[l] * 2);
        alloc((void**)&s->Y[l], npix * kCout[l] * 2);
        if (l < kLayers - 1) alloc((void**)&s->Z[l], npix * kCout[l] * 2);
    }
    if (!okm) {
        cudaGetLastError();
        free_sur(s);
        delete s;
        return VLBM_ENOMEM;
    }
    // seeded initialisation: uniform(-a, a), a = sqrt(6 / fan_in) over the real input
    // channels; the padded input channels of layer 1 and outputs of layer 5 (beyond
    // `channels`) are 0, and layer 5 starts at a tenth of that scale so that the first
    // increments are small
    std::vector<float> h(off, 0.0f);
    uint64_t st = seed;
    for (int l = 0; l < kLayers; ++l) {
        const int real_in = l == 0 ? n_in : kCin[l], real_out = l == kLayers - 1 ? channels : kCout[l];
        const float a = std::sqrt(6.0f / (9.0f * real_in)) * (l == kLayers - 1 ? 0.1f : 1.0f);
        for (int co = 0; co < kCout[l]; ++co)
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < kCin[l]; ++ci) {
                    const float r = (float)((splitmix64(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.0f - 1.0f;
                    h[s->off_w[l] + ((long long)co * 9 + t) * kCin[l] + ci] = (co < real_out && ci < real_in) ? a * r : 0.0f;
                }
    }
    int rc = VLBM_OK;
    if (cudaMemcpyAsync(s->params, h.data(), off * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->adam_m, 0, off * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->adam_v, 0, off * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->zero_bias, 0, 64 * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->err, 0, sizeof(int), s->stream) != cudaSuccess)
        rc = VLBM_ECUDA;
    if (!rc) rc = refresh_all(s);
    if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = VLBM_ECUDA;
    if (rc) {
        free_sur(s);
        delete s;
        return rc;
    }
    *out = s;
    return VLBM_OK;
}

extern "C" void vlbm_sur_destroy(vlbm_sur* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_sur(s);
    delete s;
}

extern "C" int64_t vlbm_sur_num_params(const vlbm_sur* s) { return s ? s->nparams : 0; }

extern "C" int vlbm_sur_forward(vlbm_sur* s, const float* u, float* du, int32_t batch) {
    if (!s || !u || !du || batch < 1 || batch > s->maxB) return VLBM_EINVAL;
    int rc = sur_forward(s, u, batch, false);
    if (rc) return rc;
    const long long plane = (long long)s->H * s->W, npix = plane * batch;
    ChanScale one{};
    for (int c = 0; c < 16; ++c) one.v[c] = 1.0f;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_unpack_output<<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(s->Y[kLayers - 1], nullptr, du, one,
                                                                            plane, npix, s->C);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_sur_set_scaling(vlbm_sur* s, const float* in_scale, const float* out_scale) {
    if (!s) return VLBM_EINVAL;
    for (int c = 0; c < s->n_in; ++c) {
        const float a = in_scale ? in_scale[c] : 1.0f;
        if (!std::isfinite(a)) return VLBM_EINVAL;
        s->in_scale.v[c] = a;
    }
    for (int c = 0; c < s->C; ++c) {
        const float b = out_scale ? out_scale[c] : 1.0f;
        if (!std::isfinite(b)) return VLBM_EINVAL;
        s->out_scale.v[c] = b;
    }
    return VLBM_OK;
}

extern "C" int vlbm_sur_set_train_noise(vlbm_sur* s, const float* sigma, uint64_t seed) {
    if (!s) return VLBM_EINVAL;
    ChanScale h{};
    bool any = false;
    for (int c = 0; c < s->n_in; ++c) {
        const float v = sigma ? sigma[c] : 0.0f;
        if (!(v >= 0.0f) || !std::isfinite(v)) return VLBM_EINVAL;
        h.v[c] = v;
        any = any || v > 0.0f;
    }
    if (cudaMemcpyAsync(s->noise_dev, &h, sizeof(h), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return VLBM_ECUDA;
    s->use_noise = any;
    s->noise_seed = seed;
    s->noise_draws = 0;
    return VLBM_OK;
}

extern "C" int vlbm_sur_increment(vlbm_sur* s, const float* u, float* du, int32_t batch) {
    if (!s || !u || !du || batch < 1 || batch > s->maxB || du == u) return VLBM_EINVAL;
    int rc = sur_forward(s, u, batch, false);
    if (rc) return rc;
    const long long plane = (long long)s->H * s->W, npix = plane * batch;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (s->features & VLBM_SUR_FEATURE_CURL)
        k_unpack_curl<<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(s->Y[kLayers - 1], nullptr, du,
                                                                              s->out_scale, s->H, s->W, npix, s->C);
    else
        k_unpack_output<<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(s->Y[kLayers - 1], nullptr, du,
                                                                                s->out_scale, plane, npix, s->C);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_sur_advance(vlbm_sur* s, const float* u, float* u_next, int32_t batch) {
    if (!s || !u || !u_next || batch < 1 || batch > s->maxB) return VLBM_EINVAL;
    int rc = sur_forward(s, u, batch, false);
    if (rc) return rc;
    const long long plane = (long long)s->H * s->W, npix = plane * batch;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (s->features & VLBM_SUR_FEATURE_CURL) {
        if (u_next == u) return VLBM_EINVAL;     // the curl reads neighbours of the output's source
        k_unpack_curl<<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(s->Y[kLayers - 1], u, u_next,
                                                                              s->out_scale, s->H, s->W, npix, s->C);
    } else {
        k_unpack_output<<<(unsigned)((npix + 255) / 256), 256, 0, s->stream>>>(s->Y[kLayers - 1], u, u_next,
                                                                                s->out_scale, plane, npix, s->C);
    }
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_field_pool(const float* in, float* out, int64_t B, int64_t C, int64_t H, int64_t W, int32_t factor,
                               void* stream) {
    if (!in || !out || B < 1 || C < 1 || H < 1 || W < 1 || factor < 1) return VLBM_EINVAL;
    const long long n = B * C * H * W;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_pool<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, out, n, (int)H, (int)W, factor);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_sur_gather_pairs(const float* snaps, const int64_t* idx, float* u, float* target,
                                     int32_t channels, int64_t H, int64_t W, int32_t batch, const float* inv_scale,
                                     void* stream) {
    if (!snaps || !idx || !u || !target || !inv_scale || channels < 1 || channels > 16 || H < 1 || W < 1 || batch < 1)
        return VLBM_EINVAL;
    ChanScale inv{};
    for (int c = 0; c < channels; ++c) inv.v[c] = inv_scale[c];
    const long long n = (long long)channels * H * W * batch;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_gather_pairs<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(snaps, idx, u, target, H * W,
                                                                                   channels, batch, inv);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_field_diff_norms(const float* a, const float* b, double* out, int32_t nfields, int64_t n,
                                     int64_t ld, void* stream) {
    if (!a || !b || !out || nfields < 1 || nfields > 65535 || n < 1 || ld < n) return VLBM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(out, 0, sizeof(double) * 2 * nfields, st) != cudaSuccess) return VLBM_ECUDA;
    const unsigned gx = (unsigned)std::min<long long>((n + 255) / 256, 148);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_diff_norms<<<dim3(gx, nfields), 256, 0, st>>>(a, b, out, n, ld);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_field_stats(const float* u, double* out, int32_t batch, int32_t channels, int64_t H, int64_t W,
                                void* stream) {
    if (!u || !out || batch < 1 || batch > 65535 || channels < 2 || H < 1 || W < 1 || H * W >= (1ll << 31))
        return VLBM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(out, 0, sizeof(double) * 3 * batch, st) != cudaSuccess) return VLBM_ECUDA;
    const long long plane = H * W;
    const unsigned gx = (unsigned)std::min<long long>((plane + 255) / 256, 148);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_field_stats<<<dim3(gx, batch), 256, 0, st>>>(u, out, channels, (int)H, (int)W);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_sur_rollout_check(const double* stats, const double* prev, const double* e0, const double* r_max,
                                      int32_t n, double step_tol, double drift_tol, uint8_t* mask, int64_t* counts,
                                      void* stream) {
    if (!stats || !prev || !e0 || !r_max || !mask || !counts || n < 1) return VLBM_EINVAL;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_rollout_check<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        stats, prev, e0, r_max, n, step_tol, drift_tol, mask, reinterpret_cast<unsigned long long*>(counts));
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

extern "C" int vlbm_sur_train_step(vlbm_sur* s, const float* u, const float* target, int32_t batch, float lr,
                                   float* loss) {
    if (!s || !u || !target || batch < 1 || batch > s->maxB) return VLBM_EINVAL;
    const long long plane = (long long)s->H * s->W, npix = plane * batch;
    int rc = sur_forward(s, u, batch, true);
    if (rc) return rc;
    if (cudaMemsetAsync(s->sse, 0, sizeof(double), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->grads, 0, s->nparams * 4, s->stream) != cudaSuccess)
        return VLBM_ECUDA;
    const unsigned eb = (unsigned)((npix + 255) / 256);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (s->features & VLBM_SUR_FEATURE_CURL) {
        k_curl_residual<<<eb, 256, 0, s->stream>>>(s->Y[kLayers - 1], target, s->resid, s->sse, s->H, s->W, npix,
                                                   s->C);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        k_curl_grad<<<eb, 256, 0, s->stream>>>(s->resid, s->dA, s->H, s->W, npix, s->C,
                                               1.0f / (float)((long long)s->C * npix));
    } else {
        k_mse_grad<<<eb, 256, 0, s->stream>>>(s->Y[kLayers - 1], target, s->dA, s->sse, plane, npix,
                                              1.0f / (float)((long long)s->C * npix), s->C);
    }
    // backward, last layer first: dA holds dZ of layer l (its pre-activation gradient)
    for (int l = kLayers - 1; l >= 0; --l) {
        const void* xin = l == 0 ? (const void*)s->X0 : (const void*)s->Y[l - 1];
        rc = wgrad_any(kCin[l], kCout[l], xin, s->dA, s->grads + s->off_w[l], s->grads + s->off_b[l], batch, s->H,
                       s->W, s->err, s->stream);
        if (rc) return rc;
        if (l == 0) break;
        // dY of layer l-1 = conv(dZ_l, flipped transposed W_l); then dZ_{l-1} = dY * GELU'(Z_{l-1})
        rc = conv_any(kCout[l], kCin[l], s->dA, s->Wflip[l], s->zero_bias, s->dB, nullptr, batch, s->H, s->W, 0,
                      s->err, s->stream);
        if (rc) return rc;
        const long long n = npix * kCin[l];
        g_launches.fetch_add(1, std::memory_order_relaxed);
        k_gelu_back<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(s->dB, s->Z[l - 1], s->dA, n);
    }
    s->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)s->adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)s->adam_t));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    k_adam<<<(unsigned)((s->nparams + 255) / 256), 256, 0, s->stream>>>(s->params, s->adam_m, s->adam_v, s->grads,
                                                                         s->nparams, lr, b1, b2, 1e-8f, c1, c2);
    rc = refresh_all(s);
    if (rc) return rc;
    if (loss) {
        double h = 0.0;
        if (cudaMemcpyAsync(&h, s->sse, sizeof(double), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            return VLBM_ECUDA;
        rc = check_err(s);
        if (rc) return rc;
        *loss = (float)(h / (double)((long long)s->C * npix));
    }
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}

static int copy_vec(vlbm_sur* s, void* dst, const void* src, long long n) {
    if (cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDefault, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return VLBM_ECUDA;
    return VLBM_OK;
}

extern "C" int vlbm_sur_get_params(vlbm_sur* s, float* dst) {
    return (!s || !dst) ? VLBM_EINVAL : copy_vec(s, dst, s->params, s->nparams);
}
extern "C" int vlbm_sur_get_grads(vlbm_sur* s, float* dst) {
    return (!s || !dst) ? VLBM_EINVAL : copy_vec(s, dst, s->grads, s->nparams);
}
extern "C" int vlbm_sur_set_params(vlbm_sur* s, const float* src) {
    if (!s || !src) return VLBM_EINVAL;
    int rc = copy_vec(s, s->params, src, s->nparams);
    if (rc) return rc;
    s->adam_t = 0;
    if (cudaMemsetAsync(s->adam_m, 0, s->nparams * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->adam_v, 0, s->nparams * 4, s->stream) != cudaSuccess)
        return VLBM_ECUDA;
    rc = refresh_all(s);
    if (rc) return rc;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? VLBM_OK : VLBM_ECUDA;
}
extern "C" int vlbm_sur_status(vlbm_sur* s) { return s ? check_err(s) : VLBM_EINVAL; }

extern "C" int64_t vlbm_sur_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
