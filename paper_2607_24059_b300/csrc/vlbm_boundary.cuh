// Ghost-cell boundary conditions of a 2D channel (Section 6.2.1) for the uniform FP64 / FP32
// layouts: the domain [0, n_x dx] x [0, n_y dx] with
//   left  side (x = -dx/2):     prescribed velocity u_in(y), density extrapolated linearly,
//   right side (x = L_x + dx/2): prescribed pressure potential Phi_out, momentum extrapolated,
//   lower and upper walls:       zero velocity, density extrapolated.
// Each step the conserved moments of the ghost cells are formed from the interior cells of the
// current time level (collision conserves them, so the stored post-relaxation populations give
// them), and the one population of each ghost cell that streams into the domain is set to the
// ghost cell's equilibrium (Eqs. BCPoiseuilleLeftEquilibrium, BCPoiseuilleRightEquilibrium,
// BCPoiseuilleLowerEquilibrium).  With the wall correction, the wall ghosts' populations also
// get the non-equilibrium part of the same population at the adjacent interior cell
// (Eq. BCPoiseuilleLowerEquilibriumPlusCorrection).  Then every node pulls as in the periodic
// kernel, reading the ghost population where its source lies outside the domain.
//
// In the deviation variables of the kernels (g = f - F, F the rest equilibrium f^eq(rho_bar, 0),
// moments dr = rho - rho_bar and Q = dx q) the formulas read
//   left:  dr_g = 2 dr(0) - dr(1),              Q_g = (2 rho_bar dx u_in(y), 0) - Q(0)
//   right: dr_g = 2 rho_bar dx^2 Phi_out - dr(n_x - 1),  Q_g = 2 Q(n_x - 1) - Q(n_x - 2)
//   walls: dr_g = 2 dr(0) - dr(1),              Q_g = -Q(0)      (rows 0, 1; n_y - 1, n_y - 2)
// (the right side's density is the linearised relation rho = rho_bar (1 + dx^2 Phi) of the
// paper's boundary formula); F cancels in every difference, so the ghost population is
// e(dr_g, Q_g) in the same deviation units as the lattice.
#pragma once

#include "vlbm_kernels_2d.cuh"

namespace vlbm {

// Ghost populations: ghost[(side * 3 + f) * n_ghost + j], side 0 left (+x entering, j = y),
// 1 right (-x, j = y), 2 lower (+y, j = x), 3 upper (-y, j = x); n_ghost = max(n_x, n_y).
template <class C>
struct ChannelBC {
    const double* u_in;     // n_y inflow velocities (device)
    C* ghost;
    int n_ghost;
    C phi_term;             // 2 rho_bar dx^2 Phi_out
    C u_scale;              // 2 rho_bar dx
    int correction;         // 1: non-equilibrium correction at the walls
};

template <class S, class C>
__device__ __forceinline__ void cell_state(const Layout<S, false, 5>& L, long long node, const Coef<C>& k,
                                           C (&g)[15], C& dr, C& Qx, C& Qy) {
#pragma unroll
    for (int p = 0; p < 15; ++p) g[p] = load_pop(L, p / 5, p % 5, node, k);
    moments_d2q5(g, dr, Qx, Qy);
}

// One thread per boundary cell; blockIdx.y = side.
template <class S>
__global__ void __launch_bounds__(kThreads)
k_channel_ghosts(const char* __restrict__ fin_b, int nx, int ny, long long plane, Coef<typename Storage<S>::C> k,
                 ChannelBC<typename Storage<S>::C> bc) {
    using C = typename Storage<S>::C;
    const Layout<S, false, 5> fin{const_cast<char*>(fin_b), plane};
    const int side = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int len = side < 2 ? ny : nx;
    if (j >= len) return;
    // the adjacent interior cell a and the next one b along the inward normal
    long long a, b;
    int l;   // the entering velocity
    switch (side) {
        case 0: a = (long long)j * nx; b = a + 1; l = 1; break;
        case 1: a = (long long)j * nx + nx - 1; b = a - 1; l = 2; break;
        case 2: a = j; b = (long long)nx + j; l = 3; break;
        default: a = (long long)(ny - 1) * nx + j; b = (long long)(ny - 2) * nx + j; l = 4; break;
    }
    if ((side < 2 && nx < 2) || (side >= 2 && ny < 2)) b = a;   // one cell across: no extrapolation partner
    C ga[15], gb[15], dra, qxa, qya, drb, qxb, qyb;
    cell_state<S>(fin, a, k, ga, dra, qxa, qya);
    cell_state<S>(fin, b, k, gb, drb, qxb, qyb);
    C dr, qx, qy;
    if (side == 0) {
        dr = C(2) * dra - drb;
        qx = bc.u_scale * (C)bc.u_in[j] - qxa;
        qy = -qya;
    } else if (side == 1) {
        dr = bc.phi_term - dra;
        qx = C(2) * qxa - qxb;
        qy = C(2) * qya - qyb;
    } else {
        dr = C(2) * dra - drb;
        qx = -qxa;
        qy = -qya;
    }
    C e[15];
    equilibrium_d2q5<C, false>(k, dr, qx, qy, e);
    C ea[15];
    const bool corr = side >= 2 && bc.correction;
    if (corr) equilibrium_d2q5<C, false>(k, dra, qxa, qya, ea);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        C v = e[5 * f + l];
        if (corr) v += ga[5 * f + l] - ea[5 * f + l];
        bc.ghost[(long long)(side * 3 + f) * bc.n_ghost + j] = v;
    }
}

// The stream-collide step of a channel, one thread per node: the periodic per-node body with the
// pull of each population that would cross a side replaced by that side's ghost population.
template <class S>
__global__ void __launch_bounds__(kThreads)
k_stream_collide_2d_channel(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny,
                            long long plane, Coef<typename Storage<S>::C> k,
                            ChannelBC<typename Storage<S>::C> bc, uint32_t* __restrict__ step_ctr, int par) {
    using C = typename Storage<S>::C;
    using L = Layout<S, false, 5>;
    constexpr bool SR = StochasticMoments<S>::value;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const uint32_t key = take_step_key(step_ctr, par);
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= plane) return;
    const int x = (int)(node % nx), y = (int)(node / nx);
    const long long row = (long long)y * nx;
    const C* gh = bc.ghost;
    const long long ng = bc.n_ghost;
    C g[15];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        g[5 * f] = load_pop(fin, f, 0, node, k);
        g[5 * f + 1] = x == 0 ? gh[(0 * 3 + f) * ng + y] : load_pop(fin, f, 1, row + x - 1, k);
        g[5 * f + 2] = x == nx - 1 ? gh[(1 * 3 + f) * ng + y] : load_pop(fin, f, 2, row + x + 1, k);
        g[5 * f + 3] = y == 0 ? gh[(2 * 3 + f) * ng + x] : load_pop(fin, f, 3, node - nx, k);
        g[5 * f + 4] = y == ny - 1 ? gh[(3 * 3 + f) * ng + x] : load_pop(fin, f, 4, node + nx, k);
    }
    C dr, Qx, Qy;
    moments_d2q5(g, dr, Qx, Qy);
    relax_d2q5<C, false, SR>(k, g, dr, Qx, Qy, SR ? sr_node_word(key, node) : 0u);
#pragma unroll
    for (int p = 0; p < 15; ++p) store_pop(fout, p / 5, p % 5, node, g[p], k);
}

}  // namespace vlbm
