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
// 16-bit formats also convert two values at once with stochastic rounding
// (PTX cvt.rs, sm_100a/sm_103a): `hi` takes its random bits from r[31:16], `lo`
// from r[15:0]; the result packs hi in the upper and lo in the lower half.
template <> struct Storage<__half> {
    using C = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float to_c(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from_c(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ __half from_bits(uint32_t b) { return __ushort_as_half((unsigned short)b); }
    // two packed values (element 0 in the low half) to a float pair and back, rounding to nearest
    static __device__ __forceinline__ float2 unpack2(uint32_t w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ uint32_t pack2(float2 v) {
        const __half2 h = __float22half2_rn(v);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
    static __device__ __forceinline__ uint32_t pack2_sr(float lo, float hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};
template <> struct Storage<__nv_bfloat16> {
    using C = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_c(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_bits(uint32_t b) {
        return __ushort_as_bfloat16((unsigned short)b);
    }
    // a bfloat16 is the upper half of the binary32 with the same value
    static __device__ __forceinline__ float2 unpack2(uint32_t w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ uint32_t pack2(float2 v) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
    static __device__ __forceinline__ uint32_t pack2_sr(float lo, float hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};

// Storage whose moment-carrying populations are rounded stochastically in the
// compute type: FP32 (the compute type is the storage type).  FP64 keeps
// round-to-nearest; 16-bit storage rounds at its own conversion.
template <class S> struct StochasticMoments { static constexpr bool value = std::is_same<S, float>::value; };
// 16-bit shifted storage, whose rest populations can be rounded stochastically at their
// conversion (Coef::sr16, off by default).
template <class S> struct StochasticStore16 {
    static constexpr bool value = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
};

// ---------------------------------------------------------------- index division
// n / d for 32-bit unsigned n by one multiply-high: with M = ceil(2^64 / d), floor(M n / 2^64)
// is exactly floor(n / d) for every 32-bit n and d (Lemire, Kaser and Kurz, "Faster remainder
// by direct computation", 2019).  The kernels split a warp's work item into (segment, row, plane)
// with it instead of 64-bit division.  d = 1 keeps M = 0 and returns n.
struct FastDiv {
    uint32_t d;
    unsigned long long M;
    static FastDiv make(uint32_t d) {
        return FastDiv{d, d <= 1 ? 0ull : ~0ull / d + 1ull};
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        return M ? (uint32_t)__umul64hi(M, (unsigned long long)n) : n;
    }
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
    C scale[kMaxFields];   // stored = g * scale_k (1 for unscaled formats)
    C inv_scale[kMaxFields];
    C i2m;                 // 1 / (2 mu)
    C rho_bar;
    C p_bar;               // P(rho_bar) = rho_bar^gamma
    C gamma;
    int gamma_one;         // gamma == 1: dP = dr / (2 mu) exactly
    int sr16;              // shifted 16-bit storage: rest populations rounded stochastically (else to nearest)
    // The same coefficients in stored units, al_s = alpha scale_k and i2m_s = scale_0 / (2 mu): every
    // term of a moving equilibrium is linear in (alpha, 1/(2 mu)), so equilibria built on them come
    // out multiplied by the storage scale (the split layouts use one scale for every field, 1/dx^2)
    // and can be combined with stored non-equilibrium parts without converting them.
    C al_s[kMaxFields];
    C i2m_s;
    // Single-precision pairs (both halves equal) for the paired FP32 instructions of the split
    // kernels, which update two nodes per instruction: al_s, -4 al_s (2D rest weight, exact),
    // 1 - omega_k, -(1 - omega_k) al_s, i2m_s, rho_bar and 1 / scale.
    float2 p_al[kMaxFields], p_nal4[kMaxFields], p_w[kMaxFields], p_nwal[kMaxFields];
    float2 p_i2m, p_rho_bar, p_inv_s;
};

// Coefficient selection: deviation units, or stored units (Coef::al_s, i2m_s).
template <bool STORED, class C>
__device__ __forceinline__ C coef_alpha(const Coef<C>& k, int f) { return STORED ? k.al_s[f] : k.al[f]; }
template <bool STORED, class C>
__device__ __forceinline__ C coef_i2m(const Coef<C>& k) { return STORED ? k.i2m_s : k.i2m; }

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

// ---------------------------------------------------------------- stochastic rounding
// Under the parabolic scaling dt = dx^2 / mu a conserved moment changes by a
// tiny amount per step: on a 4096^2 shear layer about one FP32 ulp of the
// population that carries it, and less than half an ulp away from the layer
// core.  Round-to-nearest then drops (or doubles) the same fraction of the
// increment at every step, a bias that grows linearly with the step count.
// The populations that carry a field's moment (the rest populations of the
// uniform layouts, the moments of the split layouts) are therefore rounded
// stochastically in FP32 storage: the exact sum a + b is rounded to the
// neighbouring float on either side with probabilities proportional to the
// distances (unbiased; the accumulated error grows like the square root of
// the step count).  The random words come from a counter-based hash of
// (node, field, step): runs are bitwise reproducible, independent of the
// launch shape and of graph replay.

// 32-bit integer finaliser (a multiply-xorshift hash with the constants of
// C. Wellons' "hash prospector" low-bias 32-bit search): a bijection of
// uint32 with good avalanche.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x21f0aaadu;
    x ^= x >> 15;
    x *= 0x735a2d97u;
    x ^= x >> 15;
    return x;
}

// Per-launch key of time step `step`.
__device__ __forceinline__ uint32_t sr_step_key(uint32_t step) { return mix32(step * 0x9e3779b9u + 0x632be5abu); }

// Random word of field f at a node: one hash per node, the fields offset by the
// 32-bit golden-ratio constant (each word is uniform; the fields' decisions act
// on independent fractional parts).
__device__ __forceinline__ uint32_t sr_node_word(uint32_t key, long long node) {
    return mix32((uint32_t)node ^ key ^ mix32((uint32_t)((unsigned long long)node >> 32)));
}
__device__ __forceinline__ uint32_t sr_field_word(uint32_t w, int f) { return w + (uint32_t)f * 0x9e3779b9u; }

// a + b rounded stochastically to FP32 with the random word r: the result is
// the round-to-nearest sum s or its neighbour t on the side of the exact
// remainder e = (a + b) - s (TwoSum), t with probability |e| / |t - s|.
__device__ __forceinline__ float sr_add(float a, float b, uint32_t r) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const uint32_t bits = __float_as_uint(s);
    // the low 31 bits are the magnitude: +1 moves away from zero, -1 toward it
    const uint32_t tb = ((__float_as_uint(e) ^ bits) >> 31) ? bits - 1u : bits + 1u;
    const float t = __uint_as_float(tb);
    const float gap = fabsf(__fsub_rn(t, s));                    // a power of two
    const float u = __uint2float_rz(r >> 8) * 0x1p-24f;         // uniform in [0, 1), 24 bits
    return fabsf(e) > __fmul_rn(u, gap) ? t : s;                 // false when e = 0 or s is not finite
}
// FP64 storage keeps round-to-nearest (its rounding is 2^-29 of FP32's).
__device__ __forceinline__ double sr_add(double a, double b, uint32_t) { return a + b; }

// 16-bit shifted storage: the rest population of field f of nodes (2j, 2j + 1)
// is converted as one pair with the random word of the even node; one node
// alone (the per-node kernels) takes the same bits of the same word.
template <class S>
__device__ __forceinline__ S sr16_store_one(float v, long long node, uint32_t key, int f) {
    const uint32_t r = sr_field_word(sr_node_word(key, node & ~1LL), f);
    const uint32_t d = (node & 1) ? (Storage<S>::pack2_sr(0.0f, v, r) >> 16) : (Storage<S>::pack2_sr(v, 0.0f, r) & 0xffffu);
    return Storage<S>::from_bits(d);
}

// Equilibrium deviations g^eq of one D2Q5 node, fields (rho, q_x, q_y) x
// velocities (rest, +x, -x, +y, -y): e[5k + l].
// STORED: the moving entries in stored units (coef_alpha / coef_i2m); the rest entries are then not
// meaningful (the split kernels do not use them).
template <class C, bool APPROX = false, bool STORED = false>
__device__ __forceinline__ void equilibrium_d2q5(const Coef<C>& k, C dr, C Qx, C Qy, C (&e)[15]) {
    const C i2m = coef_i2m<STORED>(k);
    const C r = recip_sel<APPROX>(k.rho_bar + dr);
    const C dP = pressure_dev(k, dr) * i2m;
    const C hx = Qx * i2m, hy = Qy * i2m;
    const C xx = Qx * Qx * r * i2m;
    const C xy = Qx * Qy * r * i2m;
    const C yy = Qy * Qy * r * i2m;
    // rest entries m - 4 (alpha m): the moving entries' alpha m, so the entries sum to m
    const C ar = coef_alpha<STORED>(k, 0) * dr;
    e[0] = dr - C(4) * ar;
    e[1] = ar + hx;
    e[2] = ar - hx;
    e[3] = ar + hy;
    e[4] = ar - hy;
    const C ax = coef_alpha<STORED>(k, 1) * Qx;
    e[5] = Qx - C(4) * ax;
    e[6] = ax + (xx + dP);
    e[7] = ax - (xx + dP);
    e[8] = ax + xy;
    e[9] = ax - xy;
    const C ay = coef_alpha<STORED>(k, 2) * Qy;
    e[10] = Qy - C(4) * ay;
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
// For the rest population the increment e_0 - g_0 = (1 - 2D alpha) m - g_0 is
// formed as s - 2D (alpha m) with s the moving sum (same value, since
// m = g_0 + s): it is small, while (1 - 2D alpha) m and g_0 are both of the size
// of m, and their difference would keep only the rounding of the first.  The
// product alpha m is the one the moving equilibria are built on, so that the
// relaxation conserves the moment exactly in real arithmetic for the stored
// coefficients; a separately rounded rest weight 1 - 2D alpha would differ from
// 1 - 2D alpha_stored by up to half an ulp of 1 and create or destroy moment at a
// fixed relative rate every step.
// SR: the rest population (which carries the field's moment) is rounded
// stochastically with the node's random word w (FP32 storage).
template <class C, bool APPROX = false, bool SR = false>
__device__ __forceinline__ void relax_d2q5(const Coef<C>& k, C (&g)[15], C dr, C Qx, C Qy, uint32_t w = 0) {
    C e[15];
    equilibrium_d2q5<C, APPROX>(k, dr, Qx, Qy, e);
    const C m[3] = {dr, Qx, Qy};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        C* h = g + 5 * f;
        const C d0 = moving_sum_d2q5(h) - C(4) * (k.al[f] * m[f]);
        h[0] = SR ? sr_add(h[0], k.om[f] * d0, sr_field_word(w, f)) : fma(k.om[f], d0, h[0]);
#pragma unroll
        for (int l = 1; l < 5; ++l) h[l] = fma(k.om[f], e[5 * f + l] - h[l], h[l]);
    }
}

// Equilibrium deviations of one D3Q7 node, fields (rho, q_x, q_y, q_z) x
// velocities (rest, +x, -x, +y, -y, +z, -z): e[7k + l].  The paper gives the
// 2D equilibria and states that 3D follows from the Cartesian structure; this
// is the direction-by-direction extension (rest weight 1 - 6 alpha).
template <class C, bool APPROX = false, bool STORED = false>
__device__ __forceinline__ void equilibrium_d3q7(const Coef<C>& k, C dr, const C (&Q)[3], C (&e)[28]) {
    const C i2m = coef_i2m<STORED>(k);
    const C r = recip_sel<APPROX>(k.rho_bar + dr);
    const C dP = pressure_dev(k, dr) * i2m;
    const C ar = coef_alpha<STORED>(k, 0) * dr;
    e[0] = dr - C(6) * ar;   // m - 6 (alpha m), as in 2D
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const C h = Q[d] * i2m;
        e[1 + 2 * d] = ar + h;
        e[2 + 2 * d] = ar - h;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const C a = coef_alpha<STORED>(k, j + 1) * Q[j];
        const C qr = Q[j] * r * i2m;
        e[7 * (j + 1)] = Q[j] - C(6) * a;
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
template <class C, bool APPROX = false, bool SR = false>
__device__ __forceinline__ void relax_d3q7(const Coef<C>& k, C (&g)[28], C dr, const C (&Q)[3], uint32_t w = 0) {
    C e[28];
    equilibrium_d3q7<C, APPROX>(k, dr, Q, e);
    const C m[4] = {dr, Q[0], Q[1], Q[2]};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        C* h = g + 7 * f;
        const C d0 = moving_sum_d3q7(h) - C(6) * (k.al[f] * m[f]);
        h[0] = SR ? sr_add(h[0], k.om[f] * d0, sr_field_word(w, f)) : fma(k.om[f], d0, h[0]);
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

// Loads of lattice data.  A step kernel reads the level it does not write, so its loads take the
// read-only (non-coherent) path; a kernel that runs several steps writes in one step what it
// reads in the next (COH): those loads bypass L1 and read L2 (ld.global.cg), which is coherent
// within the kernel once the step boundary's barrier has ordered the writes before them.
template <bool COH, class T>
__device__ __forceinline__ T ld_lattice(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ __half ld_lattice(const __half* p) {
    const unsigned short b = ld_lattice<COH>(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_half(b);
}
template <bool COH>
__device__ __forceinline__ __nv_bfloat16 ld_lattice(const __nv_bfloat16* p) {
    const unsigned short b = ld_lattice<COH>(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(b);
}

// A plain load, or the coherent one of a multi-step kernel.
template <bool COH, class T>
__device__ __forceinline__ T ld_plain(const T* p) {
    if constexpr (COH) return ld_lattice<true>(p);
    else return *p;
}

template <class S, int V, bool COH = false>
__device__ __forceinline__ void vload(S (&e)[V], const S* p) {
    using R = typename RawVec<V * sizeof(S)>::T;
    *reinterpret_cast<R*>(&e[0]) = ld_lattice<COH>(reinterpret_cast<const R*>(p));
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
    __device__ __forceinline__ Acc fold() const { return *this; }
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

// ---------------------------------------------------------------- paired single precision
// Blackwell executes two independent FP32 additions, multiplications or fused multiply-adds
// in one instruction (FADD2 / FMUL2 / FFMA2, each half rounded to nearest as its scalar
// form).  Every node of a lane runs the same arithmetic, so the instruction-bound kernels
// (the split steps, the fused diagnostics) let nodes (2p, 2p + 1) of a lane share each
// instruction.  The helpers below have a scalar and a pair overload with the same rounding,
// so one template body serves the pairs and the lone halo nodes of the warp edges, and a
// node's outgoing populations come out bit for bit the same whichever lane computes them.
__device__ __forceinline__ float p_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float p_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float p_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float p_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float p_neg(float a) { return -a; }
__device__ __forceinline__ float p_rcp(float x) { return recip_sel<true>(x); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, p_neg(b)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_rcp(float2 x) { return make_float2(recip_sel<true>(x.x), recip_sel<true>(x.y)); }

// A coefficient as the operand type: its scalar, or its pre-duplicated pair.
template <class T> __device__ __forceinline__ T p_coef(float c, float2 c2);
template <> __device__ __forceinline__ float p_coef<float>(float c, float2) { return c; }
template <> __device__ __forceinline__ float2 p_coef<float2>(float, float2 c2) { return c2; }

// Accumulators of the node-pair kernels: the even and odd node of each pair keep their own
// (hi, lo) pairs in the two halves of a float2, updated by the paired FP32 instructions
// (FADD2: two additions, each rounded to nearest, in one instruction) with the same TwoSum
// as Acc; fold() merges the halves into an Acc before the warp and block trees.
struct AccPair {
    float2 hi[5], lo[5];
    float mx, bad;
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 5; ++i) hi[i] = lo[i] = make_float2(0.0f, 0.0f);
        mx = bad = 0.0f;
    }
    __device__ __forceinline__ void add(int i, float2 x) {   // TwoSum, as two_sum_acc
        const float2 s = p_add(hi[i], x);
        const float2 bb = p_sub(s, hi[i]);
        lo[i] = p_add(lo[i], p_add(p_sub(hi[i], p_sub(s, bb)), p_sub(x, bb)));
        hi[i] = s;
    }
    __device__ __forceinline__ Acc<float> fold() const {
        Acc<float> a;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            a.hi[i] = hi[i].x;
            a.lo[i] = lo[i].x + lo[i].y;
            two_sum_acc(a.hi[i], a.lo[i], hi[i].y);
        }
        a.mx = mx;
        a.bad = bad;
        return a;
    }
};

// Accumulator type of a kernel: node pairs for FP32 compute, single nodes for FP64.
template <class C> struct AccOf { using T = Acc<C>; };
template <> struct AccOf<float> { using T = AccPair; };

// accumulate_node for the two nodes of a pair (dr, Q as float pairs).  0 * v is 0 for a finite
// v and NaN otherwise, so z flags a node with a non-finite moment; such a node is counted in
// `bad` and enters every sum as 0 (as accumulate_node skips it).
__device__ __forceinline__ void accumulate_pair(AccPair& acc, float2 dr, const float2* Q, int dim, float rho_bar) {
    const float2 zero = make_float2(0.0f, 0.0f);
    float2 z = p_mul(dr, zero);
    for (int d = 0; d < dim; ++d) z = p_fma(Q[d], zero, z);
    float2 q[3] = {zero, zero, zero};
    for (int d = 0; d < dim; ++d) q[d] = Q[d];
    if (!(z.x == 0.0f && z.y == 0.0f)) {
        const bool f0 = z.x == 0.0f, f1 = z.y == 0.0f;
        acc.bad += (f0 ? 0.0f : 1.0f) + (f1 ? 0.0f : 1.0f);
        dr = make_float2(f0 ? dr.x : 0.0f, f1 ? dr.y : 0.0f);
        for (int d = 0; d < dim; ++d) q[d] = make_float2(f0 ? q[d].x : 0.0f, f1 ? q[d].y : 0.0f);
    }
    const float2 rho = p_add(make_float2(rho_bar, rho_bar), dr);
    const float2 r = make_float2(recip(rho.x), recip(rho.y));
    float2 q2 = p_mul(q[0], q[0]);
    for (int d = 1; d < dim; ++d) q2 = p_fma(q[d], q[d], q2);
    acc.add(0, dr);
    for (int d = 0; d < dim; ++d) acc.add(1 + d, q[d]);
    acc.add(4, p_mul(p_mul(make_float2(0.5f, 0.5f), q2), r));
    const float2 u2 = p_mul(p_mul(q2, r), r);
    acc.mx = fmaxf(acc.mx, fmaxf(u2.x, u2.y));
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

// The 8 invariants from the folded sums s = { sum dr, sum Q_d (3), sum |Q|^2/(2 rho),
// max |Q|/rho, bad, 0 }: { N rho_bar + sum dr, sum Q_d / dx (3), E_kin, max|u|,
// non-finite nodes, sum dr }.  scale_e = dx^(d-2) turns sum |Q|^2/(2 rho) into
// 1/2 sum |q|^2/rho dx^d.
__device__ __forceinline__ void write_invariants(double* __restrict__ out, const double* s, double nodes,
                                                 double rho_bar, double inv_dx, double scale_e) {
    out[0] = nodes * rho_bar + s[0];
    out[1] = s[1] * inv_dx;
    out[2] = s[2] * inv_dx;
    out[3] = s[3] * inv_dx;
    out[4] = s[4] * scale_e;
    out[5] = s[5] * inv_dx;
    out[6] = s[6];
    out[7] = s[0];
}

// Where a fused-diagnostics step puts its invariants.  Every block writes its partial
// row, then takes a ticket on its group's counter; the last block of a group folds the
// group's rows (in row order) into stage[group], the last group folds the stage rows
// (in order) into the 8 invariants at `out`.  The folds run in a fixed order whichever
// block finishes last, so the result is deterministic, and no reduction kernel follows
// the step.  The counters return to zero by the end of the launch.
struct DiagSink {
    double* partials;          // [nblocks][8]
    double* stage;             // [ngroups][8]
    unsigned int* counters;    // [ngroups + 1], zero before the launch
    double* out;               // 8 doubles
    int nblocks, group, ngroups;
    double nodes, rho_bar, inv_dx, scale_e;
};

// Fold rows [first, first + count) of 8 doubles (sums, slot 5 a maximum) in a fixed
// order with the 256 threads of the block; thread 0 returns the 8 results in res.
// Rows written by other blocks are read past L1 (ld.global.cg).
__device__ __forceinline__ void fold_rows(const double* rows, int first, int count, double (&res)[8]) {
    __shared__ double sh[256];
    const int t = threadIdx.x, slot = t & 7;
    const bool is_max = slot == 5;
    double a = 0.0;
    for (int r = (t >> 3); r < count; r += 32) {
        const double v = __ldcg(rows + (size_t)(first + r) * 8 + slot);
        a = is_max ? fmax(a, v) : a + v;
    }
    sh[t] = a;
    __syncthreads();
    for (int stride = 16; stride > 0; stride >>= 1) {
        if ((t >> 3) < stride) {
            const double o = sh[t + stride * 8];
            sh[t] = is_max ? fmax(sh[t], o) : sh[t] + o;
        }
        __syncthreads();
    }
    if (t == 0)
        for (int i = 0; i < 8; ++i) res[i] = sh[i];
    __syncthreads();
}

// block_reduce_store, then the two-level fold of DiagSink (blocks of 256 threads).
template <class C>
__device__ __forceinline__ void block_reduce_finish(Acc<C>& acc, const DiagSink& sink) {
    __shared__ int s_last;
    block_reduce_store(acc, sink.partials);   // thread 0 writes this block's row
    const int g = (int)blockIdx.x / sink.group;
    const int gsize = min(sink.group, sink.nblocks - g * sink.group);
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(sink.counters + g, 1u) == (unsigned int)(gsize - 1);
    }
    __syncthreads();
    if (!s_last) return;
    double res[8];
    fold_rows(sink.partials, g * sink.group, gsize, res);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) sink.stage[(size_t)g * 8 + i] = res[i];
        sink.counters[g] = 0u;
        __threadfence();
        s_last = atomicAdd(sink.counters + sink.ngroups, 1u) == (unsigned int)(sink.ngroups - 1);
    }
    __syncthreads();
    if (!s_last) return;
    fold_rows(sink.stage, 0, sink.ngroups, res);
    if (threadIdx.x == 0) {
        write_invariants(sink.out, res, sink.nodes, sink.rho_bar, sink.inv_dx, sink.scale_e);
        sink.counters[sink.ngroups] = 0u;
    }
}

}  // namespace vlbm
