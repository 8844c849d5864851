// D3Q7 vectorial step kernels (4 fields x 7 velocities = 28 populations per node):
// fused transport + relaxation (the field kernels are in vlbm_fields.cuh).  Layout: 28 planes addressed through
// Layout<S, SPLIT, 7>, each plane n_z x n_y x n_x, x fastest; velocities rest,
// +x, -x, +y, -y, +z, -z.
#pragma once

#include "vlbm_kernels_2d.cuh"

namespace vlbm {

// Nodes per lane in 3D: at most 2 (28 planes x V values stay in registers):
// 8-byte vectors for FP32, 4-byte for the 16-bit formats, one FP64 per lane.
template <class S> struct Vec8 {
    static constexpr int V = (8 / sizeof(S)) < 2 ? (8 / sizeof(S)) : 2;
};

// Resident blocks per SM the register budget is bounded for: the FP32 and 16-bit plain steps
// fit 80 registers (three blocks; the 16-bit ones with every load first, 40.2 -> 49.8 GLUPS
// for FP16 at 256^3); the steps with fused diagnostics 128 (two; unbounded, they took
// 184-203 registers and ran one block per SM).  FP64 keeps the compiler's choice.
template <class S, bool DIAG>
constexpr int blocks_3d() { return sizeof(S) == 8 ? 1 : (DIAG ? 2 : 3); }

// Fused stream-collide, vectorised along x (n_x % V == 0).  Warp w handles
// 32 V consecutive nodes of one (y, z) row.  x-shifts by warp shuffle as in
// 2D; +-y are rows y -+ 1 of the same z slab, +-z the same row of slab z -+ 1.
template <class S, bool SPLIT, bool DIAG>
__global__ void __launch_bounds__(kThreads, blocks_3d<S, DIAG>())
k_stream_collide_3d_vec(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, int nz,
                        long long plane, int warps_per_row, Coef<typename Storage<S>::C> k,
                        DiagSink sink, uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, SPLIT, 7>;
    using R = typename L::R;
    constexpr int V = Vec8<S>::V;
    constexpr bool SR = StochasticMoments<S>::value && !SPLIT;
    constexpr bool SR16 = StochasticStore16<S>::value && !SPLIT;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint32_t key = take_step_key(step_ctr, par);
    typename AccOf<C>::T acc;   // node pairs for FP32 compute (V = 2)
    if (DIAG) acc.zero();
    // (64-bit division here: the multiply-high split of the 2D kernels cost this kernel
    // registers, a larger spill and 16 % of its FP32 throughput)
    for (long long item = gwarp, items = (long long)ny * nz * warps_per_row; item < items; item += (DIAG ? nwarps : items)) {   // warp-uniform
        const long long r = item / warps_per_row;         // row index (z * ny + y)
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int x0 = ((int)(item % warps_per_row) * 32 + lane) * V;
        const bool active = x0 < nx;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        const long long row = r * nx;
        const long long src_row[7] = {row, row, row, ((long long)z * ny + ym) * nx, ((long long)z * ny + yp) * nx,
                                      ((long long)zm * ny + y) * nx, ((long long)zp * ny + y) * nx};
        const int xm = x0 == 0 ? nx - 1 : x0 - 1;
        const int xp = x0 + V >= nx ? 0 : x0 + V;
        const bool fetch_next = active && (lane == 31 || x0 + V >= nx);

        C g[28][V];
        // 16-bit storage: every vector of the lane and the warp-edge elements requested before the
        // first shuffle (half the bytes per warp of FP32 need more of them in flight), also in the
        // persistent loop of the recorded step (FP16 at 256^3: 823 -> 412 us per recorded step,
        // 120 registers); FP32, at the HBM roofline with either order, keeps the interleaved one
        constexpr bool LOAD_FIRST = sizeof(S) == 2;
        if constexpr (LOAD_FIRST) {
            R raw0[4][V];
            S raw[4][6][V];
            S edge_l[4], edge_r[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                load_or_zero<R, V>(raw0[f], fin.rest(f) + row + x0, active);
#pragma unroll
                for (int l = 1; l < 7; ++l) load_or_zero<S, V>(raw[f][l - 1], fin.mov(f, l) + src_row[l] + x0, active);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                edge_l[f] = edge_r[f] = Storage<S>::from_c(C(0));
                if (lane == 0 && active) edge_l[f] = __ldg(fin.mov(f, 1) + row + xm);
                if (fetch_next) edge_r[f] = __ldg(fin.mov(f, 2) + row + xp);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const C risc = rest_load_scale<S, SPLIT>(k, f);
                const C isc = mov_load_scale<S>(k, f);
#pragma unroll
                for (int i = 0; i < V; ++i) g[7 * f][i] = Storage<R>::to_c(raw0[f][i]) * risc;
                {
                    S prev = __shfl_up_sync(0xffffffffu, raw[f][0][V - 1], 1);
                    if (lane == 0) prev = edge_l[f];
                    g[7 * f + 1][0] = Storage<S>::to_c(prev) * isc;
#pragma unroll
                    for (int i = 1; i < V; ++i) g[7 * f + 1][i] = Storage<S>::to_c(raw[f][0][i - 1]) * isc;
                }
                {
                    S next = __shfl_down_sync(0xffffffffu, raw[f][1][0], 1);
                    if (fetch_next) next = edge_r[f];
#pragma unroll
                    for (int i = 0; i < V - 1; ++i) g[7 * f + 2][i] = Storage<S>::to_c(raw[f][1][i + 1]) * isc;
                    g[7 * f + 2][V - 1] = Storage<S>::to_c(next) * isc;
                }
#pragma unroll
                for (int l = 3; l < 7; ++l)
#pragma unroll
                    for (int i = 0; i < V; ++i) g[7 * f + l][i] = Storage<S>::to_c(raw[f][l - 1][i]) * isc;
            }
        } else
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const C risc = rest_load_scale<S, SPLIT>(k, f);
            const C isc = mov_load_scale<S>(k, f);
            {
                R w[V];
                load_or_zero<R, V>(w, fin.rest(f) + row + x0, active);
#pragma unroll
                for (int i = 0; i < V; ++i) g[7 * f][i] = Storage<R>::to_c(w[i]) * risc;
            }
#pragma unroll
            for (int l = 1; l < 7; ++l) {
                const S* pl = fin.mov(f, l);
                S w[V];
                load_or_zero<S, V>(w, pl + src_row[l] + x0, active);
                if (l == 1) {           // +x: from x - 1
                    S prev = __shfl_up_sync(0xffffffffu, w[V - 1], 1);
                    if (lane == 0 && active) prev = __ldg(pl + row + xm);
                    g[7 * f + 1][0] = Storage<S>::to_c(prev) * isc;
#pragma unroll
                    for (int i = 1; i < V; ++i) g[7 * f + 1][i] = Storage<S>::to_c(w[i - 1]) * isc;
                } else if (l == 2) {    // -x: from x + 1
                    S next = __shfl_down_sync(0xffffffffu, w[0], 1);
                    if (fetch_next) next = __ldg(pl + row + xp);
#pragma unroll
                    for (int i = 0; i < V - 1; ++i) g[7 * f + 2][i] = Storage<S>::to_c(w[i + 1]) * isc;
                    g[7 * f + 2][V - 1] = Storage<S>::to_c(next) * isc;
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) g[7 * f + l][i] = Storage<S>::to_c(w[i]) * isc;
                }
            }
        }

        C mom[4][V];   // moments of the transported populations, for the diagnostics
#pragma unroll
        for (int i = 0; i < V; ++i) {
            C gn[28];
#pragma unroll
            for (int p = 0; p < 28; ++p) gn[p] = g[p][i];
            C dr, Q[3];
            moments_d3q7(gn, dr, Q);
            if constexpr (DIAG) {
                mom[0][i] = dr;
#pragma unroll
                for (int d = 0; d < 3; ++d) mom[1 + d][i] = Q[d];
                if constexpr (!std::is_same<decltype(acc), AccPair>::value) {
                    if (active) accumulate_node(acc, moments_finite(dr, Q, 3), dr, Q, 3, k.rho_bar);
                }
            }
            relax_d3q7<C, sizeof(S) == 2, SR>(k, gn, dr, Q, SR ? sr_node_word(key, row + x0 + i) : 0u);
#pragma unroll
            for (int p = 0; p < 28; ++p) g[p][i] = gn[p];
        }
        if constexpr (DIAG && std::is_same<decltype(acc), AccPair>::value) {
            static_assert(V == 2, "one node pair per lane");
            if (active) {
                const float2 Q[3] = {make_float2(mom[1][0], mom[1][1]), make_float2(mom[2][0], mom[2][1]),
                                     make_float2(mom[3][0], mom[3][1])};
                accumulate_pair(acc, make_float2(mom[0][0], mom[0][1]), Q, 3, k.rho_bar);
            }
        }

        if (active) {
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                {
                    const C rsc = rest_store_scale<S, SPLIT>(k, f);
                    R w[V];
                    bool sr16 = false;
                    if constexpr (SR16) {
                        sr16 = k.sr16 != 0;   // uniform over the launch
                        if (sr16) {   // pairs of nodes, stochastic rounding (V is even)
#pragma unroll
                            for (int j = 0; j < V / 2; ++j) {
                                const uint32_t r = sr_field_word(sr_node_word(key, row + x0 + 2 * j), f);
                                const uint32_t d =
                                    Storage<S>::pack2_sr(g[7 * f][2 * j] * rsc, g[7 * f][2 * j + 1] * rsc, r);
                                w[2 * j] = Storage<S>::from_bits(d & 0xffffu);
                                w[2 * j + 1] = Storage<S>::from_bits(d >> 16);
                            }
                        }
                    }
                    if (!sr16) {
#pragma unroll
                        for (int i = 0; i < V; ++i) w[i] = Storage<R>::from_c(g[7 * f][i] * rsc);
                    }
                    vstore<R, V>(fout.rest(f) + row + x0, w);
                }
                const C sc = mov_store_scale<S>(k, f);
#pragma unroll
                for (int l = 1; l < 7; ++l) {
                    S w[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) w[i] = Storage<S>::from_c(g[7 * f + l][i] * sc);
                    vstore<S, V>(fout.mov(f, l) + row + x0, w);
                }
            }
        }
    }
    if (DIAG) {
        Acc<C> a = acc.fold();
        block_reduce_finish(a, sink);
    }
}

// One thread per node, any size.
template <class S, bool SPLIT, bool DIAG>
__global__ void __launch_bounds__(kThreads)
k_stream_collide_3d_generic(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, int nz,
                            long long plane, Coef<typename Storage<S>::C> k, DiagSink sink,
                            uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, SPLIT, 7>;
    constexpr bool SR = StochasticMoments<S>::value && !SPLIT;
    constexpr bool SR16 = StochasticStore16<S>::value && !SPLIT;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const uint32_t key = take_step_key(step_ctr, par);
    Acc<C> acc;
    if (DIAG) acc.zero();
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < plane;
         node += (DIAG ? (long long)gridDim.x * blockDim.x : plane)) {
        const int x = (int)(node % nx);
        const long long r = node / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        const long long src[7] = {node,
                                  r * nx + xm,
                                  r * nx + xp,
                                  ((long long)z * ny + ym) * nx + x,
                                  ((long long)z * ny + yp) * nx + x,
                                  ((long long)zm * ny + y) * nx + x,
                                  ((long long)zp * ny + y) * nx + x};
        C g[28];
#pragma unroll
        for (int p = 0; p < 28; ++p) g[p] = load_pop(fin, p / 7, p % 7, src[p % 7], k);
        C dr, Q[3];
        moments_d3q7(g, dr, Q);
        if (DIAG) accumulate_node(acc, moments_finite(dr, Q, 3), dr, Q, 3, k.rho_bar);
        relax_d3q7<C, sizeof(S) == 2, SR>(k, g, dr, Q, SR ? sr_node_word(key, node) : 0u);
#pragma unroll
        for (int p = 0; p < 28; ++p) {
            if constexpr (SR16) {
                if (p % 7 == 0 && k.sr16) {
                    fout.rest(p / 7)[node] =
                        sr16_store_one<S>(g[p] * rest_store_scale<S, SPLIT>(k, p / 7), node, key, p / 7);
                    continue;
                }
            }
            store_pop(fout, p / 7, p % 7, node, g[p], k);
        }
    }
    if (DIAG) block_reduce_finish(acc, sink);
}

}  // namespace vlbm
