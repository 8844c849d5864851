// Device-side building blocks of the vectorial lattice Boltzmann update
// (Section 2 of the paper): storage traits, per-field coefficients and the
// per-node relaxation written on deviations from the rest equilibrium.
//
// Deviation variables.  Every format stores g = f - F, where F = f^eq(rho_bar, 0)
// is the (spatially uniform) rest equilibrium.  F is a fixed point of the
// relaxation and is invariant under transport, and the relaxation is affine,
// so the scheme maps g exactly as it maps f:  g* = g + omega_k (g^eq - g) with
// g^eq = f^eq(rho, q) - F.  The moments become
//     dr = rho - rho_bar = sum_l g^rho_l,     Q_d = dx q_d = sum_l g^{q_d}_l,
// and, writing r = 1/rho and i2m = 1/(2 mu), the equilibria of Section 2 read
//     rho field : rest (1 - 2D a_r) dr,     +-e_d : a_r dr +- i2m Q_d
//     q_j field : rest (1 - 2D a_j) Q_j,    +-e_d : a_j Q_j +- (i2m Q_j Q_d r + delta_jd dP)
// with dP = (P(rho) - P(rho_bar)) / (2 mu).  Nothing here depends on dx: it
// only enters through the moments' scale.  All quantities are O(perturbation),
// so FP32 keeps full relative precision of the pressure signal even when
// rho - rho_bar = O(dx^2) (the raw populations of a momentum field carry the
// constant +-P(rho_bar)/(2 mu), which would swamp it).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace vlbm {

constexpr int kMaxFields = 4;

// ---------------------------------------------------------------- storage traits
template <class S> struct Storage;
template <> struct Storage<double> {
    using C = double;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ double to_c(double v) { return v; }
    static __device__ __forceinline__ double from_c(double v) { return v; }
};
template <> struct Storage<float> {
    using C = float;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ float to_c(float v) { return v; }
    static __device__ __forceinline__ float from_c(float v) { return v; }
};
template <> struct Storage<__half> {
    using C = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float to_c(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from_c(float v) { return __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    using C = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_c(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- lattice layout
// Plane addressing of one population lattice of F = (Q + 1) / 2 fields x Q
// velocities over N nodes (a plane holds one population of every node, x fastest).
//   uniform (SPLIT = false): F * Q planes of S, plane k * Q + l.
//   mixed   (SPLIT = true):  the F rest planes (l = 0) in FP32, then the
//                            F * (Q - 1) moving planes of S, plane k * (Q - 1) + l - 1.
// The mixed layout keeps the population that carries each field's conserved
// moment at FP32 resolution while the moving ones use a 16-bit format.
template <class S, bool SPLIT, int Q>
struct Layout {
    static constexpr int F = (Q + 1) / 2;
    using R = typename std::conditional<SPLIT, float, S>::type;   // rest-plane storage
    char* base;
    long long N;
    __device__ __forceinline__ R* rest(int k) const {
        return SPLIT ? reinterpret_cast<R*>(base) + (long long)k * N
                     : reinterpret_cast<R*>(base) + (long long)k * Q * N;
    }
    __device__ __forceinline__ S* mov(int k, int l) const {
        return SPLIT ? reinterpret_cast<S*>(reinterpret_cast<float*>(base) + (long long)F * N) +
                           ((long long)k * (Q - 1) + (l - 1)) * N
                     : reinterpret_cast<S*>(base) + ((long long)k * Q + l) * N;
    }
};

// Bytes of one lattice in a layout (host side mirror of Layout).
inline long long layout_bytes(int elem_bytes, bool mixed, int q, long long nodes) {
    const int f = (q + 1) / 2;
    return mixed ? nodes * (f * 4LL + (long long)f * (q - 1) * elem_bytes) : nodes * f * q * (long long)elem_bytes;
}

// ---------------------------------------------------------------- coefficients
// Per-field relaxation and equilibrium coefficients in the compute type C.
template <class C>
struct Coef {
    C om[kMaxFields];      // omega_k
    C al[kMaxFields];      // alpha_k
    C rest[kMaxFields];    // 1 - 2D alpha_k
    C scale[kMaxFields];   // stored = g * scale_k (1 for unscaled formats)
    C inv_scale[kMaxFields];
    C i2m;                 // 1 / (2 mu)
    C rho_bar;
    C p_bar;               // P(rho_bar) = rho_bar^gamma
    C gamma;
    int gamma_one;         // gamma == 1: dP = dr / (2 mu) exactly
};

// Factors from stored values to deviations (load) and back (store).  Rest planes
// of the mixed layout are FP32 and unscaled.
template <class S, bool SPLIT, class C>
__device__ __forceinline__ C rest_load_scale(const Coef<C>& k, int f) {
    return (Storage<S>::kScaled && !SPLIT) ? k.inv_scale[f] : C(1);
}
template <class S, bool SPLIT, class C>
__device__ __forceinline__ C rest_store_scale(const Coef<C>& k, int f) {
    return (Storage<S>::kScaled && !SPLIT) ? k.scale[f] : C(1);
}
template <class S, class C>
__device__ __forceinline__ C mov_load_scale(const Coef<C>& k, int f) {
    return Storage<S>::kScaled ? k.inv_scale[f] : C(1);
}
template <class S, class C>
__device__ __forceinline__ C mov_store_scale(const Coef<C>& k, int f) {
    return Storage<S>::kScaled ? k.scale[f] : C(1);
}

// P(rho_bar + dr) - P(rho_bar) without cancellation.
template <class C>
__device__ __forceinline__ C pressure_dev(const Coef<C>& k, C dr) {
    if (k.gamma_one) return dr;
    return k.p_bar * expm1(k.gamma * log1p(dr / k.rho_bar));
}

// Correctly rounded reciprocal: the same value as 1 / x, without the general
// division sequence.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
// The hardware's approximate reciprocal (PTX rcp.approx.ftz.f32, about 1 ulp): one
// instruction instead of the correctly rounded sequence.  Used where APPROX is set (the
// moment-split kernels, which are bound by their arithmetic); FP64 keeps recip().
template <bool APPROX, class C>
__device__ __forceinline__ C recip_sel(C x) { return recip(x); }
template <>
__device__ __forceinline__ float recip_sel<true, float>(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Equilibrium deviations g^eq of one D2Q5 node, fields (rho, q_x, q_y) x
// velocities (rest, +x, -x, +y, -y): e[5k + l].
template <class C, bool APPROX = false>
__device__ __forceinline__ void equilibrium_d2q5(const Coef<C>& k, C dr, C Qx, C Qy, C (&e)[15]) {
    const C r = recip_sel<APPROX>(k.rho_bar + dr);
    const C dP = pressure_dev(k, dr) * k.i2m;
    const C hx = Qx * k.i2m, hy = Qy * k.i2m;
    const C xx = Qx * Qx * r * k.i2m;
    const C xy = Qx * Qy * r * k.i2m;
    const C yy = Qy * Qy * r * k.i2m;
    const C ar = k.al[0] * dr;
    e[0] = k.rest[0] * dr;
    e[1] = ar + hx;
    e[2] = ar - hx;
    e[3] = ar + hy;
    e[4] = ar - hy;
    const C ax = k.al[1] * Qx;
    e[5] = k.rest[1] * Qx;
    e[6] = ax + (xx + dP);
    e[7] = ax - (xx + dP);
    e[8] = ax + xy;
    e[9] = ax - xy;
    const C ay = k.al[2] * Qy;
    e[10] = k.rest[2] * Qy;
    e[11] = ay + xy;
    e[12] = ay - xy;
    e[13] = ay + (yy + dP);
    e[14] = ay - (yy + dP);
}

// Sum of the moving populations of one field, in opposite pairs: the +-flux
// parts of each pair cancel before they meet the other terms.
template <class C>
__device__ __forceinline__ C moving_sum_d2q5(const C* g) {
    return (g[1] + g[2]) + (g[3] + g[4]);
}

// Moments of one D2Q5 node: m_k = g_rest + (moving sum).  The rest population
// of a momentum field carries almost all of Q; adding the small moving sum to
// it last rounds once.
template <class C>
__device__ __forceinline__ void moments_d2q5(const C (&g)[15], C& dr, C& Qx, C& Qy) {
    dr = g[0] + moving_sum_d2q5(g);
    Qx = g[5] + moving_sum_d2q5(g + 5);
    Qy = g[10] + moving_sum_d2q5(g + 10);
}

// Relaxation of Eq. LBM_scheme on the deviations of one D2Q5 node, in place.
// For the rest population the increment e_0 - g_0 = rest m - g_0 is formed as
// rest s - (1 - rest) g_0 with s the moving sum (same value, since m = g_0 + s):
// it is small, while rest m and g_0 are both of the size of m, and their
// difference would keep only the rounding of rest m.  At FP32 that rounding is
// systematic for a slowly varying field and grows linearly with the steps.
template <class C, bool APPROX = false>
__device__ __forceinline__ void relax_d2q5(const Coef<C>& k, C (&g)[15], C dr, C Qx, C Qy) {
    C e[15];
    equilibrium_d2q5<C, APPROX>(k, dr, Qx, Qy, e);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        C* h = g + 5 * f;
        const C d0 = k.rest[f] * moving_sum_d2q5(h) - (C(1) - k.rest[f]) * h[0];
        h[0] = fma(k.om[f], d0, h[0]);
#pragma unroll
        for (int l = 1; l < 5; ++l) h[l] = fma(k.om[f], e[5 * f + l] - h[l], h[l]);
    }
}

// Equilibrium deviations of one D3Q7 node, fields (rho, q_x, q_y, q_z) x
// velocities (rest, +x, -x, +y, -y, +z, -z): e[7k + l].  The paper gives the
// 2D equilibria and states that 3D follows from the Cartesian structure; this
// is the direction-by-direction extension (rest weight 1 - 6 alpha).
template <class C, bool APPROX = false>
__device__ __forceinline__ void equilibrium_d3q7(const Coef<C>& k, C dr, const C (&Q)[3], C (&e)[28]) {
    const C r = recip_sel<APPROX>(k.rho_bar + dr);
    const C dP = pressure_dev(k, dr) * k.i2m;
    const C ar = k.al[0] * dr;
    e[0] = k.rest[0] * dr;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const C h = Q[d] * k.i2m;
        e[1 + 2 * d] = ar + h;
        e[2 + 2 * d] = ar - h;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const C a = k.al[j + 1] * Q[j];
        const C qr = Q[j] * r * k.i2m;
        e[7 * (j + 1)] = k.rest[j + 1] * Q[j];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const C flux = (j == d) ? (qr * Q[d] + dP) : qr * Q[d];
            e[7 * (j + 1) + 1 + 2 * d] = a + flux;
            e[7 * (j + 1) + 2 + 2 * d] = a - flux;
        }
    }
}

template <class C>
__device__ __forceinline__ C moving_sum_d3q7(const C* g) {
    return ((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]);
}

// Moments of one D3Q7 node (rest population last, as in 2D).
template <class C>
__device__ __forceinline__ void moments_d3q7(const C (&g)[28], C& dr, C (&Q)[3]) {
    dr = g[0] + moving_sum_d3q7(g);
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[j] = g[7 * (j + 1)] + moving_sum_d3q7(g + 7 * (j + 1));
}

// Relaxation of one D3Q7 node; rest-population increment formed as in relax_d2q5.
template <class C, bool APPROX = false>
__device__ __forceinline__ void relax_d3q7(const Coef<C>& k, C (&g)[28], C dr, const C (&Q)[3]) {
    C e[28];
    equilibrium_d3q7<C, APPROX>(k, dr, Q, e);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        C* h = g + 7 * f;
        const C d0 = k.rest[f] * moving_sum_d3q7(h) - (C(1) - k.rest[f]) * h[0];
        h[0] = fma(k.om[f], d0, h[0]);
#pragma unroll
        for (int l = 1; l < 7; ++l) h[l] = fma(k.om[f], e[7 * f + l] - h[l], h[l]);
    }
}

// ---------------------------------------------------------------- vector I/O
// Aligned vector load/store of V elements of S (V * sizeof(S) in {2,4,8,16} bytes).
template <int B> struct RawVec;
template <> struct RawVec<16> { using T = uint4; };
template <> struct RawVec<8> { using T = uint2; };
template <> struct RawVec<4> { using T = unsigned int; };
template <> struct RawVec<2> { using T = unsigned short; };

template <class S, int V>
__device__ __forceinline__ void vload(S (&e)[V], const S* p) {
    using R = typename RawVec<V * sizeof(S)>::T;
    *reinterpret_cast<R*>(&e[0]) = __ldg(reinterpret_cast<const R*>(p));
}

template <class S, int V>
__device__ __forceinline__ void vstore(S* p, const S (&e)[V]) {
    using R = typename RawVec<V * sizeof(S)>::T;
    *reinterpret_cast<R*>(p) = *reinterpret_cast<const R*>(&e[0]);
}

// ---------------------------------------------------------------- diagnostics
// Invariant accumulators.  B300's FP64 pipe is narrow, so per-node work stays
// in the compute type: with FP32 compute every sum is carried as an unevaluated
// float pair (hi, lo) updated by Knuth's TwoSum, which keeps about 48 bits, and
// FP64 is used only across warps and blocks.  With FP64 compute the pair
// degenerates to plain FP64 sums.  Slots:
//   s[0] sum dr, s[1..3] sum Q_d, s[4] sum |Q|^2 / (2 rho); mx = max |Q|^2 / rho^2;
//   bad = nodes with a non-finite population.
template <class C>
__device__ __forceinline__ void two_sum_acc(C& hi, C& lo, C x) {
    if (sizeof(C) == 8) {          // FP64 compute: plain sums
        hi += x;
        return;
    }
    const C s = hi + x;
    const C bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

template <class C>
struct Acc {
    C hi[5], lo[5];
    C mx, bad;
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 5; ++i) hi[i] = lo[i] = C(0);
        mx = bad = C(0);
    }
    __device__ __forceinline__ void add(int i, C x) { two_sum_acc(hi[i], lo[i], x); }
};

// A node holds a non-finite population exactly when one of its field sums is
// non-finite (NaN and inf propagate through the sum; inf - inf is NaN), so the
// test runs on the D + 1 moments instead of every population.
template <class C>
__device__ __forceinline__ bool moments_finite(C dr, const C* Q, int dim) {
    bool ok = isfinite(dr);
    for (int d = 0; d < dim; ++d) ok = ok && isfinite(Q[d]);
    return ok;
}

template <class C>
__device__ __forceinline__ void accumulate_node(Acc<C>& acc, bool finite, C dr, const C* Q, int dim, C rho_bar) {
    if (!finite) {
        acc.bad += C(1);
        return;
    }
    const C r = recip(rho_bar + dr);
    C q2 = C(0);
    acc.add(0, dr);
    for (int d = 0; d < dim; ++d) {
        acc.add(1 + d, Q[d]);
        q2 += Q[d] * Q[d];
    }
    acc.add(4, C(0.5) * q2 * r);
    acc.mx = fmax(acc.mx, q2 * r * r);
}

// Warp tree on the pairs: (h1, l1) + (h2, l2) by TwoSum of the heads.
template <class C>
__device__ __forceinline__ void warp_reduce(Acc<C>& acc) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const C oh = __shfl_xor_sync(0xffffffffu, acc.hi[i], off);
            const C ol = __shfl_xor_sync(0xffffffffu, acc.lo[i], off);
            C h = acc.hi[i], l = acc.lo[i] + ol;
            two_sum_acc(h, l, oh);
            acc.hi[i] = h;
            acc.lo[i] = l;
        }
        acc.mx = fmax(acc.mx, __shfl_xor_sync(0xffffffffu, acc.mx, off));
        acc.bad += __shfl_xor_sync(0xffffffffu, acc.bad, off);
    }
}

// Reduce a block's accumulators into partials[blockIdx.x * 8 + i] (FP64):
// { sum dr, sum Q_x, sum Q_y, sum Q_z, sum |Q|^2/(2 rho), max |Q|/rho, bad, 0 }.
// Warp trees, then one tree over the warps' results, all in the compute type
// (float pairs for FP32); thread 0 alone converts to FP64.  Fixed shuffle
// trees and warp order: deterministic for a given launch shape.
template <class C>
__device__ __forceinline__ void block_reduce_store(Acc<C>& acc, double* __restrict__ partials) {
    __shared__ C sh_hi[32][5], sh_lo[32][5], sh_mx[32], sh_bad[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce(acc);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            sh_hi[warp][i] = acc.hi[i];
            sh_lo[warp][i] = acc.lo[i];
        }
        sh_mx[warp] = acc.mx;
        sh_bad[warp] = acc.bad;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        const bool in = lane < nw;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            acc.hi[i] = in ? sh_hi[lane][i] : C(0);
            acc.lo[i] = in ? sh_lo[lane][i] : C(0);
        }
        acc.mx = in ? sh_mx[lane] : C(0);
        acc.bad = in ? sh_bad[lane] : C(0);
        warp_reduce(acc);
        if (lane == 0) {
            double* o = partials + (size_t)blockIdx.x * 8;
#pragma unroll
            for (int i = 0; i < 5; ++i) o[i] = (double)acc.hi[i] + (double)acc.lo[i];
            o[5] = (double)sqrt(acc.mx);
            o[6] = (double)acc.bad;
            o[7] = 0.0;
        }
    }
}

}  // namespace vlbm
