// D2Q5 vectorial step kernels: fused transport + relaxation (initialisation, macroscopic
// fields, invariant reductions and export are in vlbm_fields.cuh).
//
// Lattice layout in HBM (one lattice per time level, two levels ping-pong):
//   15 planes (field k = rho, q_x, q_y; velocity l = rest, +x, -x, +y, -y),
//   each plane n_y rows of n_x elements, x fastest, no padding, addressed
//   through Layout<S, SPLIT, 5> (vlbm_device.cuh).  Uniform layouts hold the
//   post-relaxation deviations g*(t) (see vlbm_device.cuh); the split layout
//   holds FP32 moments and 16-bit non-equilibrium parts (vlbm_split.cuh), and
//   its step kernels live there.
//
// One time step (pull form of the transport of Section 2):
//   g(t+dt, x) for velocity c_l is g*(t, x - c_l dx); relax it; store g*(t+dt, x).
// Each population is read once and written once: 15 reads + 15 writes per node.
#pragma once

#include "vlbm_device.cuh"

namespace vlbm {

constexpr int kThreads = 256;

// Nodes per lane of the vectorised 2D kernel: 16-byte vectors for FP32 (4) and
// FP64 (2); 8-byte vectors (4 nodes) for the 16-bit formats, so that every
// format keeps at most 15 x 4 values in registers.
template <class S> struct Vec16 {
    static constexpr int V = (16 / sizeof(S)) < 4 ? (16 / sizeof(S)) : 4;
};

template <class T, int V, bool COH = false>
__device__ __forceinline__ void load_or_zero(T (&w)[V], const T* p, bool active) {
    if (active) {
        vload<T, V, COH>(w, p);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) w[i] = Storage<T>::from_c(typename Storage<T>::C(0));
    }
}

// ------------------------------------------------------------------------------
// Fused stream-collide, vectorised.  Requires n_x % V == 0 (V nodes per lane).
// Warp w handles 32 V consecutive nodes of one row; lane L the V nodes starting
// at x0.  The +x population of node x comes from x - 1: lane L takes its own
// vector shifted by one element and the last element of lane L-1 by a warp
// shuffle (lane 0 loads that element from memory, with periodic wrap).  The
// -x population comes from x + 1, symmetrically.  +y / -y are whole rows
// y - 1 / y + 1 (periodic), loaded aligned.
// DIAG: also reduce the invariants of the transported state (time t + dt)
// into per-block FP64 partials, at no extra HBM traffic.
// One warp's share of a step on the uniform layout (plane 5k + l of N nodes at
// fin + (5k + l) N): V * 32 consecutive nodes of row y starting at segment seg.
// Called with every lane of the warp (shuffles); lanes past the row end load
// nothing and store nothing.  key: the step's stochastic-rounding key
// (sr_step_key).  LOAD_FIRST: request all fifteen vectors (and the warp-edge
// elements) before the first shuffle; otherwise each plane is shifted right after
// its load.  Measured at 4096^2: load-first is faster for one segment per warp
// (FP32 0.2948 against 0.3162 ms); inside the persistent loops of the recorded
// step and the batch kernel it is faster for the 16-bit formats, which move
// half the bytes per lane (FP16 recorded step 225 -> 187 us; batched FP16 78 ->
// 90 GLUPS), and slower for FP32 (recorded step ~360 against 324 us).
template <class S, bool DIAG, int V = Vec16<S>::V, bool LOAD_FIRST = !DIAG, bool COH = false, class A>
__device__ __forceinline__ void warp_stream_collide_2d(const S* __restrict__ fin, S* __restrict__ fout, long long N,
                                                       int nx, int ny, int y, int seg, int lane,
                                                       const Coef<typename Storage<S>::C>& k, A& acc, uint32_t key) {
    using C = typename Storage<S>::C;
    using R = S;
    constexpr bool SR = StochasticMoments<S>::value;
    constexpr bool SR16 = StochasticStore16<S>::value;
    auto in_plane = [&](int f, int l) { return fin + (long long)(5 * f + l) * N; };
    auto out_plane = [&](int f, int l) { return fout + (long long)(5 * f + l) * N; };
    {
        const int x0 = (seg * 32 + lane) * V;
        const bool active = x0 < nx;
        const long long row = (long long)y * nx;
        const long long row_m = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
        const long long row_p = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
        const int xm = x0 == 0 ? nx - 1 : x0 - 1;        // left neighbour of the lane's first node
        const int xp = x0 + V >= nx ? 0 : x0 + V;         // right neighbour of the lane's last node
        const bool fetch_next = active && (lane == 31 || x0 + V >= nx);

        C g[15][V];
        if constexpr (!LOAD_FIRST) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const C risc = rest_load_scale<S, false>(k, f);
                const C isc = mov_load_scale<S>(k, f);
                S w[V];
                load_or_zero<S, V, COH>(w, in_plane(f, 0) + row + x0, active);
#pragma unroll
                for (int i = 0; i < V; ++i) g[5 * f + 0][i] = Storage<S>::to_c(w[i]) * risc;
                const S* px = in_plane(f, 1);
                load_or_zero<S, V, COH>(w, px + row + x0, active);
                {
                    S prev = __shfl_up_sync(0xffffffffu, w[V - 1], 1);
                    if (lane == 0 && active) prev = ld_lattice<COH>(px + row + xm);
                    g[5 * f + 1][0] = Storage<S>::to_c(prev) * isc;
#pragma unroll
                    for (int i = 1; i < V; ++i) g[5 * f + 1][i] = Storage<S>::to_c(w[i - 1]) * isc;
                }
                const S* mx = in_plane(f, 2);
                load_or_zero<S, V, COH>(w, mx + row + x0, active);
                {
                    S next = __shfl_down_sync(0xffffffffu, w[0], 1);
                    if (fetch_next) next = ld_lattice<COH>(mx + row + xp);
#pragma unroll
                    for (int i = 0; i < V - 1; ++i) g[5 * f + 2][i] = Storage<S>::to_c(w[i + 1]) * isc;
                    g[5 * f + 2][V - 1] = Storage<S>::to_c(next) * isc;
                }
                load_or_zero<S, V, COH>(w, in_plane(f, 3) + row_m + x0, active);
#pragma unroll
                for (int i = 0; i < V; ++i) g[5 * f + 3][i] = Storage<S>::to_c(w[i]) * isc;
                load_or_zero<S, V, COH>(w, in_plane(f, 4) + row_p + x0, active);
#pragma unroll
                for (int i = 0; i < V; ++i) g[5 * f + 4][i] = Storage<S>::to_c(w[i]) * isc;
            }
        } else {
            // ---- load phase: every vector of the lane (15 planes) and the warp-edge elements are
            // requested before the first shuffle, so that one warp has all its loads in flight
            S raw[3][5][V];
            S edge_l[3], edge_r[3];
    #pragma unroll
            for (int f = 0; f < 3; ++f) {
                load_or_zero<S, V, COH>(raw[f][0], in_plane(f, 0) + row + x0, active);
                load_or_zero<S, V, COH>(raw[f][1], in_plane(f, 1) + row + x0, active);
                load_or_zero<S, V, COH>(raw[f][2], in_plane(f, 2) + row + x0, active);
                load_or_zero<S, V, COH>(raw[f][3], in_plane(f, 3) + row_m + x0, active);
                load_or_zero<S, V, COH>(raw[f][4], in_plane(f, 4) + row_p + x0, active);
            }
    #pragma unroll
            for (int f = 0; f < 3; ++f) {
                edge_l[f] = edge_r[f] = Storage<S>::from_c(C(0));
                if (lane == 0 && active) edge_l[f] = ld_lattice<COH>(in_plane(f, 1) + row + xm);
                if (fetch_next) edge_r[f] = ld_lattice<COH>(in_plane(f, 2) + row + xp);
            }
            // ---- shifts and conversion to deviations
    #pragma unroll
            for (int f = 0; f < 3; ++f) {
                const C risc = rest_load_scale<S, false>(k, f);
                const C isc = mov_load_scale<S>(k, f);
    #pragma unroll
                for (int i = 0; i < V; ++i) g[5 * f + 0][i] = Storage<S>::to_c(raw[f][0][i]) * risc;
                {   // +x: from x - 1
                    S prev = __shfl_up_sync(0xffffffffu, raw[f][1][V - 1], 1);
                    if (lane == 0) prev = edge_l[f];
                    g[5 * f + 1][0] = Storage<S>::to_c(prev) * isc;
    #pragma unroll
                    for (int i = 1; i < V; ++i) g[5 * f + 1][i] = Storage<S>::to_c(raw[f][1][i - 1]) * isc;
                }
                {   // -x: from x + 1
                    S next = __shfl_down_sync(0xffffffffu, raw[f][2][0], 1);
                    if (fetch_next) next = edge_r[f];
    #pragma unroll
                    for (int i = 0; i < V - 1; ++i) g[5 * f + 2][i] = Storage<S>::to_c(raw[f][2][i + 1]) * isc;
                    g[5 * f + 2][V - 1] = Storage<S>::to_c(next) * isc;
                }
                // +y: from y - 1;  -y: from y + 1
    #pragma unroll
                for (int i = 0; i < V; ++i) {
                    g[5 * f + 3][i] = Storage<S>::to_c(raw[f][3][i]) * isc;
                    g[5 * f + 4][i] = Storage<S>::to_c(raw[f][4][i]) * isc;
                }
            }
        }

        C mom[3][2];   // moments of the transported populations of the last node pair (diagnostics)
#pragma unroll
        for (int i = 0; i < V; ++i) {
            C gn[15];
#pragma unroll
            for (int p = 0; p < 15; ++p) gn[p] = g[p][i];
            C dr, Qx, Qy;
            moments_d2q5(gn, dr, Qx, Qy);
            if constexpr (DIAG) {
                mom[0][i & 1] = dr;
                mom[1][i & 1] = Qx;
                mom[2][i & 1] = Qy;
                if constexpr (std::is_same<A, AccPair>::value) {   // FP32: node pairs
                    if ((i & 1) && active) {
                        const float2 Q[2] = {make_float2(mom[1][0], mom[1][1]), make_float2(mom[2][0], mom[2][1])};
                        accumulate_pair(acc, make_float2(mom[0][0], mom[0][1]), Q, 2, k.rho_bar);
                    }
                } else if (active) {
                    const C Q[2] = {Qx, Qy};
                    accumulate_node(acc, moments_finite(dr, Q, 2), dr, Q, 2, k.rho_bar);
                }
            }
            relax_d2q5<C, sizeof(S) == 2, SR>(k, gn, dr, Qx, Qy, SR ? sr_node_word(key, row + x0 + i) : 0u);
#pragma unroll
            for (int p = 0; p < 15; ++p) g[p][i] = gn[p];
        }
        if (active) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                {
                    const C rsc = rest_store_scale<S, false>(k, f);
                    R w[V];
                    bool sr16 = false;
                    if constexpr (SR16) {
                        sr16 = k.sr16 != 0;   // uniform over the launch
                        if (sr16) {   // pairs of nodes, stochastic rounding (V is even)
#pragma unroll
                            for (int j = 0; j < V / 2; ++j) {
                                const uint32_t r = sr_field_word(sr_node_word(key, row + x0 + 2 * j), f);
                                const uint32_t d =
                                    Storage<S>::pack2_sr(g[5 * f][2 * j] * rsc, g[5 * f][2 * j + 1] * rsc, r);
                                w[2 * j] = Storage<S>::from_bits(d & 0xffffu);
                                w[2 * j + 1] = Storage<S>::from_bits(d >> 16);
                            }
                        }
                    }
                    if (!sr16) {
#pragma unroll
                        for (int i = 0; i < V; ++i) w[i] = Storage<R>::from_c(g[5 * f][i] * rsc);
                    }
                    vstore<R, V>(out_plane(f, 0) + row + x0, w);
                }
                const C sc = mov_store_scale<S>(k, f);
#pragma unroll
                for (int l = 1; l < 5; ++l) {
                    S w[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) w[i] = Storage<S>::from_c(g[5 * f + l][i] * sc);
                    vstore<S, V>(out_plane(f, l) + row + x0, w);
                }
            }
        }
    }
}

// Step counter of the stochastic rounding: a step that reads lattice level `par`
// reads its step number from step_ctr[par] and writes the next one to
// step_ctr[par ^ 1], which the following step (reading the other level) reads.
// Kernel boundaries order the accesses, so graph replay needs no host update.
__device__ __forceinline__ uint32_t take_step_key(uint32_t* __restrict__ step_ctr, int par) {
    const uint32_t step = step_ctr[par];
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) step_ctr[par ^ 1] = step + 1u;
    return sr_step_key(step);
}

// 16-bit storage moves half the bytes per node, so it needs more warps in flight to
// cover the memory latency: three resident blocks per SM (at most 85 registers); its step
// with fused diagnostics keeps eight nodes per lane at two blocks per SM (at 85 registers it
// spilled).  The FP32 step with fused diagnostics takes V = 2 nodes per lane (DiagVec), at
// three blocks per SM.
template <class S, bool DIAG> struct DiagVec { static constexpr int V = Vec16<S>::V; };
template <> struct DiagVec<float, true> { static constexpr int V = 2; };

template <class S, bool SPLIT, bool DIAG>
__global__ void __launch_bounds__(kThreads, (sizeof(S) == 2 && DIAG) ? 2 : ((sizeof(S) == 2 || (sizeof(S) == 4 && DIAG)) ? 3 : 1))
k_stream_collide_2d_vec(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, long long plane,
                        FastDiv wdiv, Coef<typename Storage<S>::C> k, DiagSink sink,
                        uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    static_assert(!SPLIT, "the split layouts have their own step kernels");
    const S* fin = reinterpret_cast<const S*>(fin_b);   // based on the __restrict__ parameters
    S* fout = reinterpret_cast<S*>(fout_b);
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t key = take_step_key(step_ctr, par);
    typename AccOf<C>::T acc;   // node pairs for FP32 compute
    if (DIAG) acc.zero();
    // one row segment per warp; a smaller (persistent) grid loops, accumulating the
    // diagnostics of all its segments before one block reduction
    const uint32_t items = (uint32_t)ny * wdiv.d;
    for (uint32_t item = gwarp; item < items; item += (DIAG ? nwarps : items)) {   // warp-uniform
        const uint32_t y = wdiv.div(item);
        warp_stream_collide_2d<S, DIAG, DiagVec<S, DIAG>::V, !DIAG || sizeof(S) == 2>(fin, fout, plane, nx, ny, (int)y,
                                                             (int)(item - y * wdiv.d), lane, k, acc, key);
    }
    if (DIAG) {
        Acc<C> a = acc.fold();
        block_reduce_finish(a, sink);
    }
}

// Load / store one population of one node through the layout (scaled to deviations).
template <bool COH = false, class S, bool SPLIT, int Q>
__device__ __forceinline__ typename Storage<S>::C load_pop(const Layout<S, SPLIT, Q>& L, int f, int l, long long node,
                                                           const Coef<typename Storage<S>::C>& k) {
    using R = typename Layout<S, SPLIT, Q>::R;
    if (l == 0) return Storage<R>::to_c(ld_plain<COH>(L.rest(f) + node)) * rest_load_scale<S, SPLIT>(k, f);
    return Storage<S>::to_c(ld_plain<COH>(L.mov(f, l) + node)) * mov_load_scale<S>(k, f);
}

template <class S, bool SPLIT, int Q>
__device__ __forceinline__ void store_pop(const Layout<S, SPLIT, Q>& L, int f, int l, long long node,
                                          typename Storage<S>::C v, const Coef<typename Storage<S>::C>& k) {
    using R = typename Layout<S, SPLIT, Q>::R;
    if (l == 0) L.rest(f)[node] = Storage<R>::from_c(v * rest_store_scale<S, SPLIT>(k, f));
    else L.mov(f, l)[node] = Storage<S>::from_c(v * mov_store_scale<S>(k, f));
}

// One node of the fused stream-collide (the per-node kernel's body; also the batched step's
// path for problems whose n_x is not a multiple of its vector width).  COH: coherent loads
// (the multi-step batched launch).
template <class S, bool SPLIT, bool DIAG, bool COH = false>
__device__ __forceinline__ void node_stream_collide_2d(const Layout<S, SPLIT, 5>& fin, const Layout<S, SPLIT, 5>& fout,
                                                       int nx, int ny, long long node,
                                                       const Coef<typename Storage<S>::C>& k,
                                                       Acc<typename Storage<S>::C>& acc, uint32_t key) {
    using C = typename Storage<S>::C;
    constexpr bool SR = StochasticMoments<S>::value && !SPLIT;
    constexpr bool SR16 = StochasticStore16<S>::value && !SPLIT;
    const int x = (int)(node % nx), y = (int)(node / nx);
    const long long row = (long long)y * nx;
    const long long src[5] = {
        node,
        row + (x == 0 ? nx - 1 : x - 1),
        row + (x == nx - 1 ? 0 : x + 1),
        (long long)(y == 0 ? ny - 1 : y - 1) * nx + x,
        (long long)(y == ny - 1 ? 0 : y + 1) * nx + x,
    };
    C g[15];
#pragma unroll
    for (int p = 0; p < 15; ++p) g[p] = load_pop<COH>(fin, p / 5, p % 5, src[p % 5], k);
    C dr, Qx, Qy;
    moments_d2q5(g, dr, Qx, Qy);
    if constexpr (DIAG) {
        const C Q[2] = {Qx, Qy};
        accumulate_node(acc, moments_finite(dr, Q, 2), dr, Q, 2, k.rho_bar);
    }
    relax_d2q5<C, sizeof(S) == 2, SR>(k, g, dr, Qx, Qy, SR ? sr_node_word(key, node) : 0u);
#pragma unroll
    for (int p = 0; p < 15; ++p) {
        if constexpr (SR16) {
            if (p % 5 == 0 && k.sr16) {
                fout.rest(p / 5)[node] =
                    sr16_store_one<S>(g[p] * rest_store_scale<S, SPLIT>(k, p / 5), node, key, p / 5);
                continue;
            }
        }
        store_pop(fout, p / 5, p % 5, node, g[p], k);
    }
}

// ------------------------------------------------------------------------------
// Fused stream-collide, one thread per node, any n_x (the ragged-size path).
template <class S, bool SPLIT, bool DIAG>
__global__ void __launch_bounds__(kThreads)
k_stream_collide_2d_generic(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny,
                            long long plane, Coef<typename Storage<S>::C> k, DiagSink sink,
                            uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, SPLIT, 5>;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const uint32_t key = take_step_key(step_ctr, par);
    Acc<C> acc;
    if (DIAG) acc.zero();
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < plane;
         node += (DIAG ? (long long)gridDim.x * blockDim.x : plane)) {
        node_stream_collide_2d<S, SPLIT, DIAG>(fin, fout, nx, ny, node, k, acc, key);
    }
    if (DIAG) block_reduce_finish(acc, sink);
}

}  // namespace vlbm
