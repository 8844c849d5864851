// D3Q7 vectorial kernels (4 fields x 7 velocities = 28 populations per node):
// fused transport + relaxation, initialisation, macroscopic fields and the
// FP64 invariant partials.  Layout: 28 planes p = 7k + l, each plane
// n_z x n_y x n_x, x fastest; velocities rest, +x, -x, +y, -y, +z, -z.
#pragma once

#include "vlbm_kernels_2d.cuh"

namespace vlbm {

// Nodes per lane in 3D: at most 2 (28 planes x V values stay in registers):
// 8-byte vectors for FP32, 4-byte for the 16-bit formats, one FP64 per lane.
template <class S> struct Vec8 {
    static constexpr int V = (8 / sizeof(S)) < 2 ? (8 / sizeof(S)) : 2;
};

// Fused stream-collide, vectorised along x (n_x % V == 0).  Warp w handles
// 32 V consecutive nodes of one (y, z) row.  x-shifts by warp shuffle as in
// 2D; +-y are rows y -+ 1 of the same z slab, +-z the same row of slab z -+ 1.
template <class S, bool DIAG>
__global__ void __launch_bounds__(kThreads)
k_stream_collide_3d_vec(const S* __restrict__ fin, S* __restrict__ fout, int nx, int ny, int nz, long long plane,
                        int warps_per_row, Coef<typename Storage<S>::C> k, double* __restrict__ partials) {
    using C = typename Storage<S>::C;
    constexpr int V = Vec8<S>::V;
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Acc<C> acc;
    if (DIAG) acc.zero();
    if (gwarp < (long long)ny * nz * warps_per_row) {
        const long long r = gwarp / warps_per_row;        // row index (z * ny + y)
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int x0 = ((int)(gwarp % warps_per_row) * 32 + lane) * V;
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
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const S* base = fin + (long long)(7 * f) * plane;
            const C isc = Storage<S>::kScaled ? k.inv_scale[f] : C(1);
#pragma unroll
            for (int l = 0; l < 7; ++l) {
                S w[V];
                if (active) vload<S, V>(w, base + l * plane + src_row[l] + x0);
                else {
#pragma unroll
                    for (int i = 0; i < V; ++i) w[i] = Storage<S>::from_c(C(0));
                }
                if (l == 1) {           // +x: from x - 1
                    S prev = __shfl_up_sync(0xffffffffu, w[V - 1], 1);
                    if (lane == 0 && active) prev = base[plane + row + xm];
                    g[7 * f + 1][0] = Storage<S>::to_c(prev) * isc;
#pragma unroll
                    for (int i = 1; i < V; ++i) g[7 * f + 1][i] = Storage<S>::to_c(w[i - 1]) * isc;
                } else if (l == 2) {    // -x: from x + 1
                    S next = __shfl_down_sync(0xffffffffu, w[0], 1);
                    if (fetch_next) next = base[2 * plane + row + xp];
#pragma unroll
                    for (int i = 0; i < V - 1; ++i) g[7 * f + 2][i] = Storage<S>::to_c(w[i + 1]) * isc;
                    g[7 * f + 2][V - 1] = Storage<S>::to_c(next) * isc;
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) g[7 * f + l][i] = Storage<S>::to_c(w[i]) * isc;
                }
            }
        }

#pragma unroll
        for (int i = 0; i < V; ++i) {
            C gn[28];
#pragma unroll
            for (int p = 0; p < 28; ++p) gn[p] = g[p][i];
            C dr, Q[3];
            moments_d3q7(gn, dr, Q);
            if (DIAG && active) accumulate_node(acc, moments_finite(dr, Q, 3), dr, Q, 3, k.rho_bar);
            relax_d3q7(k, gn, dr, Q);
#pragma unroll
            for (int p = 0; p < 28; ++p) g[p][i] = gn[p];
        }

        if (active) {
#pragma unroll
            for (int p = 0; p < 28; ++p) {
                const C sc = Storage<S>::kScaled ? k.scale[p / 7] : C(1);
                S w[V];
#pragma unroll
                for (int i = 0; i < V; ++i) w[i] = Storage<S>::from_c(g[p][i] * sc);
                vstore<S, V>(fout + (long long)p * plane + row + x0, w);
            }
        }
    }
    if (DIAG) block_reduce_store(acc, partials);
}

// One thread per node, any size.
template <class S, bool DIAG>
__global__ void __launch_bounds__(kThreads)
k_stream_collide_3d_generic(const S* __restrict__ fin, S* __restrict__ fout, int nx, int ny, int nz,
                            long long plane, Coef<typename Storage<S>::C> k, double* __restrict__ partials) {
    using C = typename Storage<S>::C;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Acc<C> acc;
    if (DIAG) acc.zero();
    if (node < plane) {
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
        for (int p = 0; p < 28; ++p) {
            const C isc = Storage<S>::kScaled ? k.inv_scale[p / 7] : C(1);
            g[p] = Storage<S>::to_c(fin[(long long)p * plane + src[p % 7]]) * isc;
        }
        C dr, Q[3];
        moments_d3q7(g, dr, Q);
        if (DIAG) accumulate_node(acc, moments_finite(dr, Q, 3), dr, Q, 3, k.rho_bar);
        relax_d3q7(k, g, dr, Q);
#pragma unroll
        for (int p = 0; p < 28; ++p) {
            const C sc = Storage<S>::kScaled ? k.scale[p / 7] : C(1);
            fout[(long long)p * plane + node] = Storage<S>::from_c(g[p] * sc);
        }
    }
    if (DIAG) block_reduce_store(acc, partials);
}

template <class S, class T>
__global__ void __launch_bounds__(kThreads)
k_init_3d(S* __restrict__ f, long long plane, const T* __restrict__ u, const T* __restrict__ phi,
          Coef<typename Storage<S>::C> k, double dx, double gamma, double rho_bar, double p_bar) {
    using C = typename Storage<S>::C;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    const double ph = phi ? (double)phi[node] : 0.0;
    const double lift = dx * dx * rho_bar * ph;
    const double dr = (gamma == 1.0) ? lift : rho_bar * expm1(log1p(lift / p_bar) / gamma);
    const double rho = rho_bar + dr;
    C Q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) Q[d] = (C)(dx * rho * (double)u[d * plane + node]);
    C e[28];
    equilibrium_d3q7(k, (C)dr, Q, e);
#pragma unroll
    for (int p = 0; p < 28; ++p) {
        const C sc = Storage<S>::kScaled ? k.scale[p / 7] : C(1);
        f[(long long)p * plane + node] = Storage<S>::from_c(e[p] * sc);
    }
}

template <class S, class T>
__global__ void __launch_bounds__(kThreads)
k_macros_3d(const S* __restrict__ f, long long plane, T* __restrict__ rho, T* __restrict__ u, T* __restrict__ phi,
            Coef<typename Storage<S>::C> k, double dx, double gamma, double rho_bar, double p_bar) {
    using C = typename Storage<S>::C;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    double m[4];
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) {
        const C isc = Storage<S>::kScaled ? k.inv_scale[fld] : C(1);
        C s = C(0);
#pragma unroll
        for (int l = 0; l < 7; ++l) s += Storage<S>::to_c(f[(long long)(7 * fld + l) * plane + node]) * isc;
        m[fld] = (double)s;
    }
    const double r = rho_bar + m[0];
    if (rho) rho[node] = (T)r;
    if (u)
        for (int d = 0; d < 3; ++d) u[d * plane + node] = (T)(m[1 + d] / (dx * r));
    if (phi) {
        const double dP = (gamma == 1.0) ? m[0] : p_bar * expm1(gamma * log1p(m[0] / rho_bar));
        phi[node] = (T)(dP / (dx * dx * rho_bar));
    }
}

template <class S>
__global__ void __launch_bounds__(kThreads)
k_invariants_3d(const S* __restrict__ f, long long plane, Coef<typename Storage<S>::C> k, double* __restrict__ partials) {
    using C = typename Storage<S>::C;
    Acc<C> acc;
    acc.zero();
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < plane;
         node += (long long)gridDim.x * blockDim.x) {
        C g[28];
#pragma unroll
        for (int p = 0; p < 28; ++p) {
            const C isc = Storage<S>::kScaled ? k.inv_scale[p / 7] : C(1);
            g[p] = Storage<S>::to_c(f[(long long)p * plane + node]) * isc;
        }
        C dr, Q[3];
        moments_d3q7(g, dr, Q);
        accumulate_node(acc, moments_finite(dr, Q, 3), dr, Q, 3, k.rho_bar);
    }
    block_reduce_store(acc, partials);
}

}  // namespace vlbm
