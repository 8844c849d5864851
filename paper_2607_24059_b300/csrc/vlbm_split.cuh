// Moment-split storage of the populations (VLBM_FP16_SPLIT / VLBM_BF16_SPLIT).
//
// Per node and field k the lattice stores
//   m_k          the conserved moment (dr = rho - rho_bar, or Q_j = dx q_j), FP32,
//                in the field's rest slot of Layout<S, true, Q>;
//   n_{k,l}      l = 1..Q-1: the non-equilibrium part g*_{k,l} - e_{k,l}(m_k) of
//                the post-relaxation moving population, 16-bit, scaled.
// The rest population is not stored: relaxation conserves m_k, so
// g*_{k,0} = e_{k,0}(m_k) - sum_l n_{k,l}.  In exact arithmetic this is the same
// state as the populations (an invertible change of variables per node), so
// the pull step below is the scheme of Section 2:
//   g_{k,l}(x)  = e_{k,l}(m(x - c_l)) + n_{k,l}(x - c_l)                (transport)
//   m'_k(x)     = m_k(x) + sum_l [g_{k,l}(x) - e_{k,l}(m(x))] - sum_l n_{k,l}(x)
//   n'_{k,l}(x) = (1 - omega_k) (g_{k,l}(x) - e_{k,l}(m'(x)))          (relaxation)
// The second line is g_{k,0} + sum_l g_{k,l} with e_{k,0}(m) = m - sum_l e_{k,l}(m),
// written so that m' is m plus a small increment (one rounding).  Why: the
// moving populations carry the equilibrium fluxes (+-Q/(2 mu) in the rho field,
// +-(Q_j Q_d / rho + delta P)/(2 mu) in the momentum fields), and a 16-bit copy
// of those corrupts pressure and momentum every step; the non-equilibrium parts
// are (1 - omega) times cell-to-cell differences of the equilibria, orders of
// magnitude smaller, and the conserved moments, whose per-step increments are
// tiny under the parabolic scaling, keep FP32 resolution.
//
// The step kernels work in stored units: every field of the split layout has
// the storage scale s = 1/dx^2, and the moving equilibria are built on the
// stored-unit coefficients (Coef::al_s, i2m_s), which gives s e; pulled
// populations, own parts and new parts are then combined and stored without
// converting each part, and only the moment increment is brought back by 1/s.
#pragma once

#include "vlbm_kernels_3d.cuh"

namespace vlbm {

// Nodes per lane of the split kernels (register budget: pulled populations of
// every moving velocity stay live until the new moments are known).
constexpr int kSplitV2 = 4;
constexpr int kSplitV3 = 2;

// Equilibrium deviations of every field along one moving velocity l (the split kernels take
// 1 / rho from the hardware's approximate reciprocal)
// (axis a = (l - 1) / 2, sign +1 for odd l) from the moments m of one node:
//   rho field  a_rho dr +- Q_a / (2 mu)
//   q_j field  a_j Q_j +- (Q_j Q_a / rho + delta_ja dP) / (2 mu)
// the same values as the l-th entries of equilibrium_d2q5 / _d3q7.
// equilibrium_dir_r takes r = 1/rho and dP of the node (one reciprocal serves every direction),
// dP in the units of the result.  STORED: stored units (s e).
template <class C, int F, int L, bool STORED = true>
__device__ __forceinline__ void equilibrium_dir_r(const Coef<C>& k, const C (&m)[F], C r, C dP, C (&e)[F]) {
    constexpr int a = (L - 1) / 2;
    const C s = (L & 1) ? C(1) : C(-1);
    const C i2m = coef_i2m<STORED>(k);
    const C Qa = m[1 + a];
    e[0] = coef_alpha<STORED>(k, 0) * m[0] + s * (Qa * i2m);
    const C qr = Qa * r * i2m;
#pragma unroll
    for (int j = 0; j < F - 1; ++j) {
        const C flux = (j == a) ? (m[1 + j] * qr + dP) : m[1 + j] * qr;
        e[1 + j] = coef_alpha<STORED>(k, 1 + j) * m[1 + j] + s * flux;
    }
}

template <class C, int F, int L, bool STORED = true>
__device__ __forceinline__ void equilibrium_dir(const Coef<C>& k, const C (&m)[F], C (&e)[F]) {
    equilibrium_dir_r<C, F, L, STORED>(k, m, recip_sel<true>(k.rho_bar + m[0]),
                                       pressure_dev(k, m[0]) * coef_i2m<STORED>(k), e);
}

template <class T, int V>
__device__ __forceinline__ void load_vec_c(typename Storage<T>::C (&out)[V], const T* p, bool active,
                                           typename Storage<T>::C scale) {
    T w[V];
    load_or_zero<T, V>(w, p, active);
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = Storage<T>::to_c(w[i]) * scale;
}

// Values at x - 1 (shift_right) and x + 1 (shift_left) of a per-lane vector of
// V consecutive nodes, taking the missing element from the neighbouring lane,
// or from memory at the warp edge (periodic wrap handled by the caller's index).
template <class C, int V>
__device__ __forceinline__ void shift_from_left(C (&out)[V], const C (&own)[V], bool edge, C edge_value) {
    C prev = __shfl_up_sync(0xffffffffu, own[V - 1], 1);
    out[0] = edge ? edge_value : prev;
#pragma unroll
    for (int i = 1; i < V; ++i) out[i] = own[i - 1];
}
template <class C, int V>
__device__ __forceinline__ void shift_from_right(C (&out)[V], const C (&own)[V], bool edge, C edge_value) {
    C next = __shfl_down_sync(0xffffffffu, own[0], 1);
#pragma unroll
    for (int i = 0; i < V - 1; ++i) out[i] = own[i + 1];
    out[V - 1] = edge ? edge_value : next;
}

// ------------------------------------------------------------------------------ 2D
// Relaxation and new moments of one D2Q5 node in split form.
//   m[3]: moments at the node; B[3][4]: pulled populations g_{k,l} (l = 1..4);
//   nown[3]: sum_l n_{k,l} of the node's own stored non-equilibrium parts.
// B, nown and the returned parts are in stored units; m is not.
// Returns the new moments in m and the new non-equilibrium parts in B.  The FP32 moments
// round to nearest: the split forms are held to the L2 gate of 1e-3, which they meet by a
// wide margin, and these kernels are bound by their instruction count (stochastic
// rounding, as in FP32 storage, would cost about a tenth of their throughput).
template <class C>
__device__ __forceinline__ void split_update_d2q5(const Coef<C>& k, C (&m)[3], C (&B)[3][4], const C (&nown)[3]) {
    // sum_l e_{k,l}(m) = 4 alpha_k m_k: the alpha m of the moving equilibria (their
    // +- fluxes cancel), so that the update conserves m for the stored coefficients
    const C inv_s = k.inv_scale[0];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const C pulled = (B[f][0] + B[f][1]) + (B[f][2] + B[f][3]);
        m[f] = m[f] + inv_s * ((pulled - C(4) * (k.al_s[f] * m[f])) - nown[f]);
    }
    C e[15];
    equilibrium_d2q5<C, true, true>(k, m[0], m[1], m[2], e);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const C w = C(1) - k.om[f];
#pragma unroll
        for (int l = 0; l < 4; ++l) B[f][l] = w * (B[f][l] - e[5 * f + 1 + l]);
    }
}

// Pulled populations of velocity l from source moments ms[3] and pulled n[3].
template <class C, int L>
__device__ __forceinline__ void pulled_d2q5(const Coef<C>& k, const C (&ms)[3], const C (&n)[3], C (&B)[3][4]) {
    C e[3];
    equilibrium_dir<C, 3, L>(k, ms, e);
#pragma unroll
    for (int f = 0; f < 3; ++f) B[f][L - 1] = e[f] + n[f];
}

// Vectorised 2D split step with V nodes per lane.  All loads of a lane are
// issued first (its moments, the moment rows y -+ 1, the six own-row and six
// pulled rows of non-equilibrium parts, and the warp-edge halo values), then
// the arithmetic runs: the kernel is limited by how many bytes are in flight.
template <class S, int V, bool DIAG>
__device__ __forceinline__ void warp_split_step_2d(const Layout<S, true, 5>& fin, const Layout<S, true, 5>& fout,
                                                   int nx, int ny, int y, int seg, int lane,
                                                   const Coef<typename Storage<S>::C>& k,
                                                   Acc<typename Storage<S>::C>& acc) {
    using C = typename Storage<S>::C;
    {
        const int x0 = (seg * 32 + lane) * V;
        const bool active = x0 < nx;
        const long long row = (long long)y * nx;
        const long long row_m = (long long)(y == 0 ? ny - 1 : y - 1) * nx;
        const long long row_p = (long long)(y == ny - 1 ? 0 : y + 1) * nx;
        const int xm = x0 == 0 ? nx - 1 : x0 - 1;
        const int xp = x0 + V >= nx ? 0 : x0 + V;
        const bool left_edge = lane == 0 && active;
        const bool right_edge = active && (lane == 31 || x0 + V >= nx);

        // ---- load phase
        float mo[3][V], mym[3][V], myp[3][V];
        S n_px[3][V], n_mx[3][V], n_py_pull[3][V], n_my_pull[3][V], n_py_own[3][V], n_my_own[3][V];
        float hm_l[3], hm_r[3];
        S hn_l[3], hn_r[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            load_or_zero<float, V>(mo[f], fin.rest(f) + row + x0, active);
            load_or_zero<float, V>(mym[f], fin.rest(f) + row_m + x0, active);
            load_or_zero<float, V>(myp[f], fin.rest(f) + row_p + x0, active);
            load_or_zero<S, V>(n_px[f], fin.mov(f, 1) + row + x0, active);
            load_or_zero<S, V>(n_mx[f], fin.mov(f, 2) + row + x0, active);
            load_or_zero<S, V>(n_py_pull[f], fin.mov(f, 3) + row_m + x0, active);
            load_or_zero<S, V>(n_my_pull[f], fin.mov(f, 4) + row_p + x0, active);
            load_or_zero<S, V>(n_py_own[f], fin.mov(f, 3) + row + x0, active);
            load_or_zero<S, V>(n_my_own[f], fin.mov(f, 4) + row + x0, active);
            hm_l[f] = hm_r[f] = 0.0f;
            hn_l[f] = hn_r[f] = Storage<S>::from_c(C(0));
            if (left_edge) {
                hm_l[f] = fin.rest(f)[row + xm];
                hn_l[f] = fin.mov(f, 1)[row + xm];
            }
            if (right_edge) {
                hm_r[f] = fin.rest(f)[row + xp];
                hn_r[f] = fin.mov(f, 2)[row + xp];
            }
        }

        // ---- arithmetic
        C m[3][V], nown[3][V], B[3][4][V];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            C a[V], b[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {   // parts stay in stored units
                m[f][i] = (C)mo[f][i];
                a[i] = Storage<S>::to_c(n_px[f][i]);
                b[i] = Storage<S>::to_c(n_mx[f][i]);
                nown[f][i] = (a[i] + b[i]) + (Storage<S>::to_c(n_py_own[f][i]) + Storage<S>::to_c(n_my_own[f][i]));
            }
            // pulled non-equilibrium parts, stashed in B until the equilibria are added
            C sh[V];
            shift_from_left<C, V>(sh, a, left_edge, Storage<S>::to_c(hn_l[f]));
#pragma unroll
            for (int i = 0; i < V; ++i) B[f][0][i] = sh[i];
            shift_from_right<C, V>(sh, b, right_edge, Storage<S>::to_c(hn_r[f]));
#pragma unroll
            for (int i = 0; i < V; ++i) {
                B[f][1][i] = sh[i];
                B[f][2][i] = Storage<S>::to_c(n_py_pull[f][i]);
                B[f][3][i] = Storage<S>::to_c(n_my_pull[f][i]);
            }
        }
        // source moments of the x neighbours by warp shuffle
        C mxl[3][V], mxr[3][V];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            shift_from_left<C, V>(mxl[f], m[f], left_edge, (C)hm_l[f]);
            shift_from_right<C, V>(mxr[f], m[f], right_edge, (C)hm_r[f]);
        }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            C e[3];
            {
                const C ms[3] = {mxl[0][i], mxl[1][i], mxl[2][i]};
                equilibrium_dir<C, 3, 1>(k, ms, e);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][0][i] += e[f];
            }
            {
                const C ms[3] = {mxr[0][i], mxr[1][i], mxr[2][i]};
                equilibrium_dir<C, 3, 2>(k, ms, e);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][1][i] += e[f];
            }
            {
                const C ms[3] = {(C)mym[0][i], (C)mym[1][i], (C)mym[2][i]};
                equilibrium_dir<C, 3, 3>(k, ms, e);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][2][i] += e[f];
            }
            {
                const C ms[3] = {(C)myp[0][i], (C)myp[1][i], (C)myp[2][i]};
                equilibrium_dir<C, 3, 4>(k, ms, e);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][3][i] += e[f];
            }
            C mi[3] = {m[0][i], m[1][i], m[2][i]};
            C Bi[3][4];
            const C ni[3] = {nown[0][i], nown[1][i], nown[2][i]};
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int l = 0; l < 4; ++l) Bi[f][l] = B[f][l][i];
            split_update_d2q5(k, mi, Bi, ni);
            if (DIAG && active) {
                const C Q[2] = {mi[1], mi[2]};
                accumulate_node(acc, moments_finite(mi[0], Q, 2), mi[0], Q, 2, k.rho_bar);
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                m[f][i] = mi[f];
#pragma unroll
                for (int l = 0; l < 4; ++l) B[f][l][i] = Bi[f][l];
            }
        }
        if (active) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                float wm[V];
#pragma unroll
                for (int i = 0; i < V; ++i) wm[i] = (float)m[f][i];
                vstore<float, V>(fout.rest(f) + row + x0, wm);
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    S w[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) w[i] = Storage<S>::from_c(B[f][l][i]);
                    vstore<S, V>(fout.mov(f, l + 1) + row + x0, w);
                }
            }
        }
    }
}

// At least two resident blocks per SM (at most 128 registers): the BF16 instantiation with
// fused diagnostics needs 131 and would otherwise run one block per SM.
template <class S, int V, bool DIAG>
__global__ void __launch_bounds__(kThreads, 2)
k_split_step_2d_vec(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, long long plane,
                    int warps_per_row, Coef<typename Storage<S>::C> k, DiagSink sink,
                    uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, true, 5>;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    take_step_key(step_ctr, par);   // keeps the step counter in step (the split forms round to nearest)
    Acc<C> acc;
    if (DIAG) acc.zero();
    for (long long item = gwarp, items = (long long)ny * warps_per_row; item < items; item += (DIAG ? nwarps : items))   // warp-uniform
        warp_split_step_2d<S, V, DIAG>(fin, fout, nx, ny, (int)(item / warps_per_row), (int)(item % warps_per_row),
                                       lane, k, acc);
    if (DIAG) block_reduce_finish(acc, sink);
}

// One thread per node, any size (2D split form).
template <class S, bool DIAG>
__global__ void __launch_bounds__(kThreads)
k_split_step_2d_generic(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny,
                        long long plane, Coef<typename Storage<S>::C> k, DiagSink sink,
                        uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, true, 5>;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    take_step_key(step_ctr, par);   // keeps the step counter in step (the split forms round to nearest)
    Acc<C> acc;
    if (DIAG) acc.zero();
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < plane;
         node += (DIAG ? (long long)gridDim.x * blockDim.x : plane)) {
        const int x = (int)(node % nx), y = (int)(node / nx);
        const long long row = (long long)y * nx;
        const long long src[5] = {
            node,
            row + (x == 0 ? nx - 1 : x - 1),
            row + (x == nx - 1 ? 0 : x + 1),
            (long long)(y == 0 ? ny - 1 : y - 1) * nx + x,
            (long long)(y == ny - 1 ? 0 : y + 1) * nx + x,
        };
        C m[3], nown[3] = {C(0), C(0), C(0)}, B[3][4];
#pragma unroll
        for (int f = 0; f < 3; ++f) m[f] = (C)fin.rest(f)[node];
#pragma unroll
        for (int l = 1; l < 5; ++l) {
            C ms[3], np[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                ms[f] = (C)fin.rest(f)[src[l]];
                np[f] = Storage<S>::to_c(fin.mov(f, l)[src[l]]);      // stored units
                nown[f] += Storage<S>::to_c(fin.mov(f, l)[node]);
            }
            if (l == 1) pulled_d2q5<C, 1>(k, ms, np, B);
            else if (l == 2) pulled_d2q5<C, 2>(k, ms, np, B);
            else if (l == 3) pulled_d2q5<C, 3>(k, ms, np, B);
            else pulled_d2q5<C, 4>(k, ms, np, B);
        }
        split_update_d2q5(k, m, B, nown);
        if (DIAG) {
            const C Q[2] = {m[1], m[2]};
            accumulate_node(acc, moments_finite(m[0], Q, 2), m[0], Q, 2, k.rho_bar);
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            fout.rest(f)[node] = (float)m[f];
#pragma unroll
            for (int l = 0; l < 4; ++l) fout.mov(f, l + 1)[node] = Storage<S>::from_c(B[f][l]);
        }
    }
    if (DIAG) block_reduce_finish(acc, sink);
}

// ------------------------------------------------------------------------------ 3D
template <class C>
__device__ __forceinline__ void split_update_d3q7(const Coef<C>& k, C (&m)[4], C (&B)[4][6], const C (&nown)[4]) {
    const C inv_s = k.inv_scale[0];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const C pulled = ((B[f][0] + B[f][1]) + (B[f][2] + B[f][3])) + (B[f][4] + B[f][5]);
        m[f] = m[f] + inv_s * ((pulled - C(6) * (k.al_s[f] * m[f])) - nown[f]);
    }
    C e[28];
    const C Q[3] = {m[1], m[2], m[3]};
    equilibrium_d3q7<C, true, true>(k, m[0], Q, e);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const C w = C(1) - k.om[f];
#pragma unroll
        for (int l = 0; l < 6; ++l) B[f][l] = w * (B[f][l] - e[7 * f + 1 + l]);
    }
}

template <class C, int L>
__device__ __forceinline__ void pulled_d3q7(const Coef<C>& k, const C (&ms)[4], const C (&n)[4], C (&B)[4][6]) {
    C e[4];
    equilibrium_dir<C, 4, L>(k, ms, e);
#pragma unroll
    for (int f = 0; f < 4; ++f) B[f][L - 1] = e[f] + n[f];
}

template <class C>
__device__ __forceinline__ void pulled_d3q7_l(const Coef<C>& k, int l, const C (&ms)[4], const C (&n)[4],
                                              C (&B)[4][6]) {
    switch (l) {
        case 1: pulled_d3q7<C, 1>(k, ms, n, B); break;
        case 2: pulled_d3q7<C, 2>(k, ms, n, B); break;
        case 3: pulled_d3q7<C, 3>(k, ms, n, B); break;
        case 4: pulled_d3q7<C, 4>(k, ms, n, B); break;
        case 5: pulled_d3q7<C, 5>(k, ms, n, B); break;
        default: pulled_d3q7<C, 6>(k, ms, n, B); break;
    }
}

// Vectorised along x with V = kSplitV3 nodes per lane: sources x -+ 1 by warp
// shuffle (memory at the warp edge), y -+ 1 rows, z -+ 1 slabs.
template <class S, bool DIAG>
__global__ void __launch_bounds__(kThreads, 3)
k_split_step_3d_vec(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, int nz,
                    long long plane, int warps_per_row, Coef<typename Storage<S>::C> k,
                    DiagSink sink, uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, true, 7>;
    constexpr int V = kSplitV3;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    take_step_key(step_ctr, par);   // keeps the step counter in step (the split forms round to nearest)
    Acc<C> acc;
    if (DIAG) acc.zero();
    for (long long item = gwarp, items = (long long)ny * nz * warps_per_row; item < items; item += (DIAG ? nwarps : items)) {   // warp-uniform
        const long long r = item / warps_per_row;
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
        const bool left_edge = lane == 0 && active;
        const bool right_edge = active && (lane == 31 || x0 + V >= nx);

        C m[4][V], nown[4][V], B[4][6][V];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            load_vec_c<float, V>(m[f], fin.rest(f) + row + x0, active, C(1));
#pragma unroll
            for (int i = 0; i < V; ++i) nown[f][i] = C(0);
        }
#pragma unroll
        for (int l = 1; l < 7; ++l) {
            C ms[4][V], np[4][V];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const float* mp = fin.rest(f);
                const S* npl = fin.mov(f, l);
                C own[V];
                load_vec_c<S, V>(own, npl + row + x0, active, C(1));   // stored units
#pragma unroll
                for (int i = 0; i < V; ++i) nown[f][i] += own[i];
                if (l == 1) {
                    C em = C(0), en = C(0);
                    if (left_edge) {
                        em = (C)mp[row + xm];
                        en = Storage<S>::to_c(npl[row + xm]);
                    }
                    shift_from_left<C, V>(ms[f], m[f], left_edge, em);
                    shift_from_left<C, V>(np[f], own, left_edge, en);
                } else if (l == 2) {
                    C em = C(0), en = C(0);
                    if (right_edge) {
                        em = (C)mp[row + xp];
                        en = Storage<S>::to_c(npl[row + xp]);
                    }
                    shift_from_right<C, V>(ms[f], m[f], right_edge, em);
                    shift_from_right<C, V>(np[f], own, right_edge, en);
                } else {
                    load_vec_c<float, V>(ms[f], mp + src_row[l] + x0, active, C(1));
                    load_vec_c<S, V>(np[f], npl + src_row[l] + x0, active, C(1));
                }
            }
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const C msi[4] = {ms[0][i], ms[1][i], ms[2][i], ms[3][i]};
                const C npi[4] = {np[0][i], np[1][i], np[2][i], np[3][i]};
                C Bi[4][6];
                pulled_d3q7_l(k, l, msi, npi, Bi);
#pragma unroll
                for (int f = 0; f < 4; ++f) B[f][l - 1][i] = Bi[f][l - 1];
            }
        }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            C mi[4] = {m[0][i], m[1][i], m[2][i], m[3][i]};
            const C ni[4] = {nown[0][i], nown[1][i], nown[2][i], nown[3][i]};
            C Bi[4][6];
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
                for (int l = 0; l < 6; ++l) Bi[f][l] = B[f][l][i];
            split_update_d3q7(k, mi, Bi, ni);
            if (DIAG && active) {
                const C Q[3] = {mi[1], mi[2], mi[3]};
                accumulate_node(acc, moments_finite(mi[0], Q, 3), mi[0], Q, 3, k.rho_bar);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                m[f][i] = mi[f];
#pragma unroll
                for (int l = 0; l < 6; ++l) B[f][l][i] = Bi[f][l];
            }
        }
        if (active) {
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                float wm[V];
#pragma unroll
                for (int i = 0; i < V; ++i) wm[i] = (float)m[f][i];
                vstore<float, V>(fout.rest(f) + row + x0, wm);
#pragma unroll
                for (int l = 0; l < 6; ++l) {
                    S w[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) w[i] = Storage<S>::from_c(B[f][l][i]);
                    vstore<S, V>(fout.mov(f, l + 1) + row + x0, w);
                }
            }
        }
    }
    if (DIAG) block_reduce_finish(acc, sink);
}

template <class S, bool DIAG>
__global__ void __launch_bounds__(kThreads)
k_split_step_3d_generic(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, int nz,
                        long long plane, Coef<typename Storage<S>::C> k, DiagSink sink,
                        uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, true, 7>;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    take_step_key(step_ctr, par);   // keeps the step counter in step (the split forms round to nearest)
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
        C m[4], nown[4], B[4][6];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            m[f] = (C)fin.rest(f)[node];
            nown[f] = C(0);
        }
#pragma unroll
        for (int l = 1; l < 7; ++l) {
            C ms[4], np[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                ms[f] = (C)fin.rest(f)[src[l]];
                np[f] = Storage<S>::to_c(fin.mov(f, l)[src[l]]);      // stored units
                nown[f] += Storage<S>::to_c(fin.mov(f, l)[node]);
            }
            pulled_d3q7_l(k, l, ms, np, B);
        }
        split_update_d3q7(k, m, B, nown);
        if (DIAG) {
            const C Q[3] = {m[1], m[2], m[3]};
            accumulate_node(acc, moments_finite(m[0], Q, 3), m[0], Q, 3, k.rho_bar);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            fout.rest(f)[node] = (float)m[f];
#pragma unroll
            for (int l = 0; l < 6; ++l) fout.mov(f, l + 1)[node] = Storage<S>::from_c(B[f][l]);
        }
    }
    if (DIAG) block_reduce_finish(acc, sink);
}

}  // namespace vlbm
