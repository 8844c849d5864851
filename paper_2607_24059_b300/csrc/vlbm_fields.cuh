// Field kernels around the step: initialisation at equilibrium from (u, phi), macroscopic
// fields, the FP64 invariant reductions, population export and the vorticity sum, for
// D2Q5 and D3Q7 and every storage format.  None of them is on the step path.
#pragma once

#include "vlbm_kernels_3d.cuh"

namespace vlbm {

// ------------------------------------------------------------------------------
// Initialisation at equilibrium: P(rho) = P(rho_bar) + dx^2 rho_bar phi,
// q = rho u, g = f^eq(rho, q) - F.  The density deviation is formed in FP64:
// gamma = 1 gives dr = dx^2 rho_bar phi exactly; otherwise
// dr = rho_bar expm1(log1p(dx^2 rho_bar phi / P(rho_bar)) / gamma).
// Equilibrium state of one node from u (planes x, y) and phi (may be NULL).
template <class S, bool SPLIT, class T>
__device__ __forceinline__ void init_node_2d(const Layout<S, SPLIT, 5>& f, long long plane, long long node,
                                             const T* __restrict__ u, const T* __restrict__ phi,
                                             const Coef<typename Storage<S>::C>& k, double dx, double gamma,
                                             double rho_bar, double p_bar) {
    using C = typename Storage<S>::C;
    const double ph = phi ? (double)phi[node] : 0.0;
    const double lift = dx * dx * rho_bar * ph;
    const double dr = (gamma == 1.0) ? lift : rho_bar * expm1(log1p(lift / p_bar) / gamma);
    const double rho = rho_bar + dr;
    const double Qx = dx * rho * (double)u[node];
    const double Qy = dx * rho * (double)u[plane + node];
    if constexpr (SPLIT) {   // moments, and no departure from equilibrium
        f.rest(0)[node] = (float)dr;
        f.rest(1)[node] = (float)Qx;
        f.rest(2)[node] = (float)Qy;
#pragma unroll
        for (int p = 0; p < 15; ++p)
            if (p % 5) f.mov(p / 5, p % 5)[node] = Storage<S>::from_c(C(0));
    } else {
        C e[15];
        equilibrium_d2q5(k, (C)dr, (C)Qx, (C)Qy, e);
#pragma unroll
        for (int p = 0; p < 15; ++p) store_pop(f, p / 5, p % 5, node, e[p], k);
    }
}

template <class S, bool SPLIT, class T>
__global__ void __launch_bounds__(kThreads)
k_init_2d(char* __restrict__ f_b, long long plane, const T* __restrict__ u, const T* __restrict__ phi,
          Coef<typename Storage<S>::C> k, double dx, double gamma, double rho_bar, double p_bar) {
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    init_node_2d<S, SPLIT, T>(Layout<S, SPLIT, 5>{f_b, plane}, plane, node, u, phi, k, dx, gamma, rho_bar, p_bar);
}

// Macroscopic fields of the state (moments of g*(t) = moments of g(t)), in FP64, or in FP32
// for FP32 output of an FP32-compute format.  rho, u (planes x, y) and phi of one node; any
// output may be NULL.
template <class S, bool SPLIT, class T>
__device__ __forceinline__ void macros_node_2d(const Layout<S, SPLIT, 5>& f, long long plane, long long node,
                                               T* __restrict__ rho, T* __restrict__ u, T* __restrict__ phi,
                                               const Coef<typename Storage<S>::C>& k, double dx, double gamma,
                                               double rho_bar, double p_bar) {
    using C = typename Storage<S>::C;
    if constexpr (std::is_same<C, float>::value && std::is_same<T, float>::value) {
        // single-precision output of single-precision compute: the moments as the step forms
        // them, one reciprocal (B300's FP64 divisions made this read-back FP64-bound)
        float m[3];
#pragma unroll
        for (int fld = 0; fld < 3; ++fld) {
            if constexpr (SPLIT) {
                m[fld] = f.rest(fld)[node];
            } else {
                const float mv = (load_pop(f, fld, 1, node, k) + load_pop(f, fld, 2, node, k)) +
                                 (load_pop(f, fld, 3, node, k) + load_pop(f, fld, 4, node, k));
                m[fld] = load_pop(f, fld, 0, node, k) + mv;
            }
        }
        const float r = (float)rho_bar + m[0];
        if (rho) rho[node] = r;
        if (u) {
            const float inv = 1.0f / ((float)dx * r);
            u[node] = m[1] * inv;
            u[plane + node] = m[2] * inv;
        }
        if (phi) {
            const double dP = (gamma == 1.0) ? (double)m[0] : p_bar * expm1(gamma * log1p((double)m[0] / rho_bar));
            phi[node] = (float)(dP / (dx * dx * rho_bar));
        }
        return;
    }
    double m[3];
#pragma unroll
    for (int fld = 0; fld < 3; ++fld) {
        if constexpr (SPLIT) {
            m[fld] = (double)f.rest(fld)[node];
        } else {
            double mv = 0.0;
#pragma unroll
            for (int l = 1; l < 5; ++l) mv += (double)load_pop(f, fld, l, node, k);
            m[fld] = (double)load_pop(f, fld, 0, node, k) + mv;
        }
    }
    const double r = rho_bar + m[0];
    if (rho) rho[node] = (T)r;
    if (u) {
        const double inv = 1.0 / (dx * r);   // one FP64 division per node
        u[node] = (T)(m[1] * inv);
        u[plane + node] = (T)(m[2] * inv);
    }
    if (phi) {
        const double dP = (gamma == 1.0) ? m[0] : p_bar * expm1(gamma * log1p(m[0] / rho_bar));
        phi[node] = (T)(dP / (dx * dx * rho_bar));
    }
}

template <class S, bool SPLIT, class T>
__global__ void __launch_bounds__(kThreads)
k_macros_2d(const char* __restrict__ f_b, long long plane, T* __restrict__ rho, T* __restrict__ u, T* __restrict__ phi,
            Coef<typename Storage<S>::C> k, double dx, double gamma, double rho_bar, double p_bar) {
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    macros_node_2d<S, SPLIT, T>(Layout<S, SPLIT, 5>{const_cast<char*>(f_b), plane}, plane, node, rho, u, phi, k, dx,
                                gamma, rho_bar, p_bar);
}

// Invariant partials over the stored lattice (no transport), grid-stride.
template <class S, bool SPLIT>
__global__ void __launch_bounds__(kThreads)
k_invariants_2d(const char* __restrict__ f_b, long long plane, Coef<typename Storage<S>::C> k,
                double* __restrict__ partials) {
    using C = typename Storage<S>::C;
    const Layout<S, SPLIT, 5> f{const_cast<char*>(f_b), plane};
    Acc<C> acc;
    acc.zero();
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < plane;
         node += (long long)gridDim.x * blockDim.x) {
        C dr, Qx, Qy;
        if constexpr (SPLIT) {
            dr = (C)f.rest(0)[node];
            Qx = (C)f.rest(1)[node];
            Qy = (C)f.rest(2)[node];
        } else {
            C g[15];
#pragma unroll
            for (int p = 0; p < 15; ++p) g[p] = load_pop(f, p / 5, p % 5, node, k);
            moments_d2q5(g, dr, Qx, Qy);
        }
        const C Q[2] = {Qx, Qy};
        accumulate_node(acc, moments_finite(dr, Q, 2), dr, Q, 2, k.rho_bar);
    }
    block_reduce_store(acc, partials);
}

// First stage of the reduction of many partial rows: block b folds rows
// b, b + gridDim.x, ... (fixed order) into stage[b * 8 + slot].  Spreads the
// FP64 additions over many SMs (B300's FP64 rate per SM is low); the final
// kernel then folds gridDim.x rows.  Thread t owns slot t % 8.
static __global__ void __launch_bounds__(256)
k_invariants_stage(const double* __restrict__ partials, int nblocks, double* __restrict__ stage) {
    __shared__ double sh[256];
    const int t = threadIdx.x, slot = t & 7;
    const bool is_max = slot == 5;
    double a = 0.0;
    for (int b = blockIdx.x + (t >> 3) * gridDim.x; b < nblocks; b += 32 * gridDim.x) {
        const double v = partials[(size_t)b * 8 + slot];
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
    if (t < 8) stage[(size_t)blockIdx.x * 8 + t] = sh[t];
}

// Final reduction of nblocks partials (one block of 1024 threads, fixed order)
// into the invariants { N rho_bar + sum dr, sum Q_d / dx (3), E_kin, max|u|,
// non-finite nodes, sum dr }.  Thread t owns slot t % 8 of blocks t / 8,
// t / 8 + 128, ...: consecutive threads read consecutive doubles.
// scale_e = dx^(d-2) turns sum |Q|^2/(2 rho) into 1/2 sum |q|^2/rho dx^d.
// Shared by 2D and 3D.
static __global__ void __launch_bounds__(1024)
k_invariants_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out, double nodes,
                   double rho_bar, double inv_dx, double scale_e) {
    __shared__ double sh[1024];
    const int t = threadIdx.x, slot = t & 7;
    const bool is_max = slot == 5;
    double a = 0.0;
#pragma unroll 16
    for (int b = t >> 3; b < nblocks; b += 128) {
        const double v = partials[(size_t)b * 8 + slot];
        a = is_max ? fmax(a, v) : a + v;
    }
    sh[t] = a;
    __syncthreads();
    for (int stride = 64; stride > 0; stride >>= 1) {
        if ((t >> 3) < stride) {
            const double o = sh[t + stride * 8];
            sh[t] = is_max ? fmax(sh[t], o) : sh[t] + o;
        }
        __syncthreads();
    }
    if (t == 0) write_invariants(out, sh, nodes, rho_bar, inv_dx, scale_e);
}

// Export populations in [p][node] order (p = q k + l): the stored deviation
// g_p, or g_p + F_p with the rest equilibrium F = f^eq(rho_bar, 0):
// rho field F = (f_rest, f_move, ..., f_move); momentum field j:
// +p_half on the population along +e_j, -p_half along -e_j, 0 elsewhere.
// Shared by 2D (Q = 5) and 3D (Q = 7).
template <class S, bool SPLIT, int Q, class T>
__global__ void __launch_bounds__(kThreads)
k_export(const char* __restrict__ f_b, long long total, long long plane, T* __restrict__ dst,
         Coef<typename Storage<S>::C> k, double f_rest, double f_move, double p_half, int deviation) {
    const Layout<S, SPLIT, Q> f{const_cast<char*>(f_b), plane};
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int p = (int)(i / plane);
    const long long node = i - (long long)p * plane;
    const int fld = p / Q, l = p % Q;
    double v;
    if constexpr (SPLIT) {   // g* = e(m) + n, rest: e_0(m) - sum of n
        using C = typename Storage<S>::C;
        C e[4 * 7];
        if constexpr (Q == 5) {
            C ev[15];
            equilibrium_d2q5(k, (C)f.rest(0)[node], (C)f.rest(1)[node], (C)f.rest(2)[node], ev);
            for (int i = 0; i < 15; ++i) e[i] = ev[i];
        } else {
            C ev[28];
            const C qv[3] = {(C)f.rest(1)[node], (C)f.rest(2)[node], (C)f.rest(3)[node]};
            equilibrium_d3q7(k, (C)f.rest(0)[node], qv, ev);
            for (int i = 0; i < 28; ++i) e[i] = ev[i];
        }
        const C isc = mov_load_scale<S>(k, fld);
        if (l == 0) {
            double sn = 0.0;
            for (int j = 1; j < Q; ++j) sn += (double)(Storage<S>::to_c(f.mov(fld, j)[node]) * isc);
            v = (double)e[fld * Q] - sn;
        } else {
            v = (double)e[fld * Q + l] + (double)(Storage<S>::to_c(f.mov(fld, l)[node]) * isc);
        }
    } else {
        v = (double)load_pop(f, fld, l, node, k);
    }
    if (!deviation) {
        if (fld == 0) v += (l == 0) ? f_rest : f_move;
        else if (l == 2 * (fld - 1) + 1) v += p_half;
        else if (l == 2 * (fld - 1) + 2) v -= p_half;
    }
    dst[i] = (T)v;
}


template <class S, bool SPLIT, class T>
__global__ void __launch_bounds__(kThreads)
k_init_3d(char* __restrict__ f_b, long long plane, const T* __restrict__ u, const T* __restrict__ phi,
          Coef<typename Storage<S>::C> k, double dx, double gamma, double rho_bar, double p_bar) {
    using C = typename Storage<S>::C;
    const Layout<S, SPLIT, 7> f{f_b, plane};
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    const double ph = phi ? (double)phi[node] : 0.0;
    const double lift = dx * dx * rho_bar * ph;
    const double dr = (gamma == 1.0) ? lift : rho_bar * expm1(log1p(lift / p_bar) / gamma);
    const double rho = rho_bar + dr;
    C Q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) Q[d] = (C)(dx * rho * (double)u[d * plane + node]);
    if constexpr (SPLIT) {   // moments, and no departure from equilibrium
        f.rest(0)[node] = (float)dr;
#pragma unroll
        for (int d = 0; d < 3; ++d) f.rest(d + 1)[node] = (float)Q[d];
#pragma unroll
        for (int p = 0; p < 28; ++p)
            if (p % 7) f.mov(p / 7, p % 7)[node] = Storage<S>::from_c(C(0));
    } else {
        C e[28];
        equilibrium_d3q7(k, (C)dr, Q, e);
#pragma unroll
        for (int p = 0; p < 28; ++p) store_pop(f, p / 7, p % 7, node, e[p], k);
    }
}

template <class S, bool SPLIT, class T>
__global__ void __launch_bounds__(kThreads)
k_macros_3d(const char* __restrict__ f_b, long long plane, T* __restrict__ rho, T* __restrict__ u, T* __restrict__ phi,
            Coef<typename Storage<S>::C> k, double dx, double gamma, double rho_bar, double p_bar) {
    const Layout<S, SPLIT, 7> f{const_cast<char*>(f_b), plane};
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    using C = typename Storage<S>::C;
    if constexpr (std::is_same<C, float>::value && std::is_same<T, float>::value) {
        // single-precision output of single-precision compute (as in 2D)
        float m[4];
#pragma unroll
        for (int fld = 0; fld < 4; ++fld) {
            if constexpr (SPLIT) {
                m[fld] = f.rest(fld)[node];
            } else {
                const float mv = ((load_pop(f, fld, 1, node, k) + load_pop(f, fld, 2, node, k)) +
                                  (load_pop(f, fld, 3, node, k) + load_pop(f, fld, 4, node, k))) +
                                 (load_pop(f, fld, 5, node, k) + load_pop(f, fld, 6, node, k));
                m[fld] = load_pop(f, fld, 0, node, k) + mv;
            }
        }
        const float r = (float)rho_bar + m[0];
        if (rho) rho[node] = r;
        if (u) {
            const float inv = 1.0f / ((float)dx * r);
            for (int d = 0; d < 3; ++d) u[d * plane + node] = m[1 + d] * inv;
        }
        if (phi) {
            const double dP = (gamma == 1.0) ? (double)m[0] : p_bar * expm1(gamma * log1p((double)m[0] / rho_bar));
            phi[node] = (float)(dP / (dx * dx * rho_bar));
        }
        return;
    }
    double m[4];
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) {
        if constexpr (SPLIT) {
            m[fld] = (double)f.rest(fld)[node];
        } else {
            double mv = 0.0;
#pragma unroll
            for (int l = 1; l < 7; ++l) mv += (double)load_pop(f, fld, l, node, k);
            m[fld] = (double)load_pop(f, fld, 0, node, k) + mv;
        }
    }
    const double r = rho_bar + m[0];
    if (rho) rho[node] = (T)r;
    if (u) {
        const double inv = 1.0 / (dx * r);   // one FP64 division per node
        for (int d = 0; d < 3; ++d) u[d * plane + node] = (T)(m[1 + d] * inv);
    }
    if (phi) {
        const double dP = (gamma == 1.0) ? m[0] : p_bar * expm1(gamma * log1p(m[0] / rho_bar));
        phi[node] = (T)(dP / (dx * dx * rho_bar));
    }
}

template <class S, bool SPLIT>
__global__ void __launch_bounds__(kThreads)
k_invariants_3d(const char* __restrict__ f_b, long long plane, Coef<typename Storage<S>::C> k,
                double* __restrict__ partials) {
    using C = typename Storage<S>::C;
    const Layout<S, SPLIT, 7> f{const_cast<char*>(f_b), plane};
    Acc<C> acc;
    acc.zero();
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < plane;
         node += (long long)gridDim.x * blockDim.x) {
        C dr, Q[3];
        if constexpr (SPLIT) {
            dr = (C)f.rest(0)[node];
#pragma unroll
            for (int d = 0; d < 3; ++d) Q[d] = (C)f.rest(d + 1)[node];
        } else {
            C g[28];
#pragma unroll
            for (int p = 0; p < 28; ++p) g[p] = load_pop(f, p / 7, p % 7, node, k);
            moments_d3q7(g, dr, Q);
        }
        accumulate_node(acc, moments_finite(dr, Q, 3), dr, Q, 3, k.rho_bar);
    }
    block_reduce_store(acc, partials);
}

// ------------------------------------------------------------------------------
// Vorticity diagnostic: per-block FP64 sums of |curl u|^2 with centred differences
// (periodic), u [dim][nz][ny][nx] FP32 (2D: nz = 1, the scalar d_x u_y - d_y u_x).
// The differences are taken in FP64 from the FP32 velocities; the caller scales by
// 1 / (2 dx)^2 and dx^d.  Used every few hundred steps, not on the step path.
static __global__ void __launch_bounds__(kThreads)
k_vorticity_sq(const float* __restrict__ u, int nx, int ny, int nz, int dim, double* __restrict__ partials) {
    __shared__ double sh[kThreads];
    const long long N = (long long)nx * ny * nz;
    double acc = 0.0;
    for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < N;
         node += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(node % nx);
        const long long r = node / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        auto U = [&](int c, int xx, int yy, int zz) {
            return (double)__ldg(u + (long long)c * N + ((long long)zz * ny + yy) * nx + xx);
        };
        if (dim == 2) {
            const double w = (U(1, xp, y, z) - U(1, xm, y, z)) - (U(0, x, yp, z) - U(0, x, ym, z));
            acc += w * w;
        } else {
            const double wx = (U(2, x, yp, z) - U(2, x, ym, z)) - (U(1, x, y, zp) - U(1, x, y, zm));
            const double wy = (U(0, x, y, zp) - U(0, x, y, zm)) - (U(2, xp, y, z) - U(2, xm, y, z));
            const double wz = (U(1, xp, y, z) - U(1, xm, y, z)) - (U(0, x, yp, z) - U(0, x, ym, z));
            acc += wx * wx + wy * wy + wz * wz;
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int stride = kThreads / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) sh[threadIdx.x] += sh[threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// One block: out[0] = scale * (sum of rows[0 .. n)), in a fixed order.
static __global__ void __launch_bounds__(kThreads)
k_sum_rows(const double* __restrict__ rows, int n, double scale, double* __restrict__ out) {
    __shared__ double sh[kThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) a += rows[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int stride = kThreads / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) sh[threadIdx.x] += sh[threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

}  // namespace vlbm
