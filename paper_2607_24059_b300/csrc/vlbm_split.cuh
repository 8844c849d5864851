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

// Plane base pointers of one split lattice, source and destination, passed to the kernels
// by value: every plane address is then a kernel parameter, and an access costs one
// multiply-add of its 32-bit node offset instead of 64-bit plane arithmetic.
template <class S, int Q>
struct SplitPlanes {
    static constexpr int F = (Q + 1) / 2;
    const float* rin[F];
    const S* min[F][Q - 1];
    float* rout[F];
    S* mout[F][Q - 1];
};

// Host side: the planes of Layout<S, true, Q> over N nodes at in and out.
template <class S, int Q>
inline SplitPlanes<S, Q> split_planes(const char* in, char* out, long long N) {
    constexpr int F = (Q + 1) / 2;
    SplitPlanes<S, Q> P;
    for (int f = 0; f < F; ++f) {
        P.rin[f] = reinterpret_cast<const float*>(in) + (long long)f * N;
        P.rout[f] = reinterpret_cast<float*>(out) + (long long)f * N;
        for (int l = 1; l < Q; ++l) {
            const long long plane = (long long)f * (Q - 1) + (l - 1);
            P.min[f][l - 1] = reinterpret_cast<const S*>(reinterpret_cast<const float*>(in) + (long long)F * N) + plane * N;
            P.mout[f][l - 1] = reinterpret_cast<S*>(reinterpret_cast<float*>(out) + (long long)F * N) + plane * N;
        }
    }
    return P;
}

// Source and destination views of SplitPlanes with Layout's rest() / mov() interface.
template <class S, int Q>
struct PlanesIn {
    const SplitPlanes<S, Q>& p;
    __device__ __forceinline__ const float* rest(int f) const { return p.rin[f]; }
    __device__ __forceinline__ const S* mov(int f, int l) const { return p.min[f][l - 1]; }
};
template <class S, int Q>
struct PlanesOut {
    const SplitPlanes<S, Q>& p;
    __device__ __forceinline__ float* rest(int f) const { return p.rout[f]; }
    __device__ __forceinline__ S* mov(int f, int l) const { return p.mout[f][l - 1]; }
};

// dP = P(rho_bar + dr) - P(rho_bar) in stored units (dr i2m_s for gamma = 1).
__device__ __forceinline__ float p_pressure(const Coef<float>& k, float dr) {
    return p_mul(k.gamma_one ? dr : pressure_dev(k, dr), k.i2m_s);
}
__device__ __forceinline__ float2 p_pressure(const Coef<float>& k, float2 dr) {
    if (k.gamma_one) return p_mul(dr, k.p_i2m);
    return p_mul(make_float2(pressure_dev(k, dr.x), pressure_dev(k, dr.y)), k.p_i2m);
}

// Moving equilibria of one D2Q5 node along one axis A (0: x, 1: y), stored units, as the
// terms shared by the +A and -A directions: e_{k,+A} = base_k + flux_k, e_{k,-A} = base_k - flux_k
// with base = alpha_s m and flux = (Q_A, Q_j Q_A / rho + delta_jA dP) i2m_s.  Only the flux is
// returned; callers fold alpha_s m into a fused multiply-add.
template <class T, int A>
__device__ __forceinline__ void fluxes_d2q5(const Coef<float>& k, T dr, T Qx, T Qy, T (&fl)[3]) {
    const T i2m = p_coef<T>(k.i2m_s, k.p_i2m);
    const T r = p_rcp(p_add(p_coef<T>(k.rho_bar, k.p_rho_bar), dr));
    const T dP = p_pressure(k, dr);
    const T Qa = A == 0 ? Qx : Qy;
    const T qr = p_mul(Qa, p_mul(r, i2m));            // Q_A i2m / rho
    fl[0] = p_mul(Qa, i2m);
    fl[1] = A == 0 ? p_fma(Qx, qr, dP) : p_mul(Qx, qr);
    fl[2] = A == 0 ? p_mul(Qy, qr) : p_fma(Qy, qr, dP);
}

// Both axes' fluxes of one node (the new equilibrium of the collision): one reciprocal, and the
// shared term Q_x Q_y / rho serves flux_x of field q_y and flux_y of field q_x.
template <class T>
__device__ __forceinline__ void fluxes_d2q5_xy(const Coef<float>& k, T dr, T Qx, T Qy, T (&fx)[3], T (&fy)[3]) {
    const T i2m = p_coef<T>(k.i2m_s, k.p_i2m);
    const T ri = p_mul(p_rcp(p_add(p_coef<T>(k.rho_bar, k.p_rho_bar), dr)), i2m);
    const T dP = p_pressure(k, dr);
    const T qxr = p_mul(Qx, ri), qyr = p_mul(Qy, ri);
    const T xy = p_mul(Qy, qxr);
    fx[0] = p_mul(Qx, i2m);
    fx[1] = p_fma(Qx, qxr, dP);
    fx[2] = xy;
    fy[0] = p_mul(Qy, i2m);
    fy[1] = xy;
    fy[2] = p_fma(Qy, qyr, dP);
}

// D3Q7 fluxes of one node along axis A: (Q_A, Q_j Q_A / rho + delta_jA dP) i2m_s.
template <class T, int A>
__device__ __forceinline__ void fluxes_d3q7(const Coef<float>& k, const T (&m)[4], T (&fl)[4]) {
    const T i2m = p_coef<T>(k.i2m_s, k.p_i2m);
    const T r = p_rcp(p_add(p_coef<T>(k.rho_bar, k.p_rho_bar), m[0]));
    const T dP = p_pressure(k, m[0]);
    const T qr = p_mul(m[1 + A], p_mul(r, i2m));
    fl[0] = p_mul(m[1 + A], i2m);
#pragma unroll
    for (int j = 0; j < 3; ++j) fl[1 + j] = j == A ? p_fma(m[1 + j], qr, dP) : p_mul(m[1 + j], qr);
}

// All three axes' D3Q7 fluxes of one node (the new equilibrium): one reciprocal, the cross
// terms Q_i Q_j / rho shared between the two axes they appear in.
template <class T>
__device__ __forceinline__ void fluxes_d3q7_all(const Coef<float>& k, const T (&m)[4], T (&fl)[3][4]) {
    const T i2m = p_coef<T>(k.i2m_s, k.p_i2m);
    const T ri = p_mul(p_rcp(p_add(p_coef<T>(k.rho_bar, k.p_rho_bar), m[0])), i2m);
    const T dP = p_pressure(k, m[0]);
    T qr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        qr[a] = p_mul(m[1 + a], ri);
        fl[a][0] = p_mul(m[1 + a], i2m);
        fl[a][1 + a] = p_fma(m[1 + a], qr[a], dP);
    }
    const T xy = p_mul(m[2], qr[0]), xz = p_mul(m[3], qr[0]), yz = p_mul(m[3], qr[1]);
    fl[0][2] = xy;
    fl[1][1] = xy;
    fl[0][3] = xz;
    fl[2][1] = xz;
    fl[1][3] = yz;
    fl[2][2] = yz;
}

// Post-relaxation populations leaving nodes with moments m and non-equilibrium parts n along
// +A (SIGN = +1) or -A (SIGN = -1), given the fluxes along A: e_{k,l}(m) + n_{k,l}, stored units.
template <class T, int F, int SIGN>
__device__ __forceinline__ void outgoing(const Coef<float>& k, const T (&m)[F], const T (&fl)[F], const T (&n)[F],
                                         T (&o)[F]) {
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const T e = p_fma(p_coef<T>(k.al_s[f], k.p_al[f]), m[f], SIGN > 0 ? fl[f] : p_neg(fl[f]));
        o[f] = p_add(e, n[f]);
    }
}

// Vectorised 2D split step with V nodes per lane (V even), the arithmetic in node pairs.
// All loads of a lane are issued first (its moments, the moment rows y -+ 1, the six own-row
// and six pulled rows of non-equilibrium parts, and the warp-edge halo values), then:
//   outgoing +x / -x populations of the lane's own nodes, shifted by one node (warp shuffle
//   across lanes; the edge lanes evaluate the halo node's population themselves), and
//   pulled +y / -y populations from the equilibria of rows y -+ 1, in either order;
//   the new moments, their equilibrium and the relaxed non-equilibrium parts (Section 2's
//   collision in the split variables).
template <class S, int V, bool DIAG, bool COH = false, class In, class Out, class A>
__device__ __forceinline__ void warp_split_step_2d(const In& fin, const Out& fout, int nx, int ny, int y, int seg,
                                                   int lane, const Coef<float>& k, A& acc) {
    static_assert(V % 2 == 0, "node pairs");
    constexpr int P = V / 2;
    using W = typename RawVec<V * sizeof(S)>::T;     // V 16-bit values
    using SW = Storage<S>;
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
    float2 mo[3][P], mym[3][P], myp[3][P];
    uint32_t n_px[3][P], n_mx[3][P], n_py_pull[3][P], n_my_pull[3][P], n_py_own[3][P], n_my_own[3][P];
    float hm_l[3], hm_r[3], hn_l[3], hn_r[3];
    auto ldm = [&](float2 (&d)[P], const float* p) {
        if (active) {
            float t[V];
            vload<float, V, COH>(t, p);
#pragma unroll
            for (int q = 0; q < P; ++q) d[q] = make_float2(t[2 * q], t[2 * q + 1]);
        } else {
#pragma unroll
            for (int q = 0; q < P; ++q) d[q] = make_float2(0.0f, 0.0f);
        }
    };
    auto ldn = [&](uint32_t (&d)[P], const S* p) {
        if (active) {
            const W w = ld_lattice<COH>(reinterpret_cast<const W*>(p));
            memcpy(&d[0], &w, sizeof(W));
        } else {
#pragma unroll
            for (int q = 0; q < P; ++q) d[q] = 0u;
        }
    };
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        ldm(mo[f], fin.rest(f) + row + x0);
        ldm(mym[f], fin.rest(f) + row_m + x0);
        ldm(myp[f], fin.rest(f) + row_p + x0);
        ldn(n_px[f], fin.mov(f, 1) + row + x0);
        ldn(n_mx[f], fin.mov(f, 2) + row + x0);
        ldn(n_py_pull[f], fin.mov(f, 3) + row_m + x0);
        ldn(n_my_pull[f], fin.mov(f, 4) + row_p + x0);
        ldn(n_py_own[f], fin.mov(f, 3) + row + x0);
        ldn(n_my_own[f], fin.mov(f, 4) + row + x0);
        hm_l[f] = hm_r[f] = hn_l[f] = hn_r[f] = 0.0f;
        if (left_edge) {
            hm_l[f] = ld_plain<COH>(fin.rest(f) + row + xm);
            hn_l[f] = SW::to_c(ld_plain<COH>(fin.mov(f, 1) + row + xm));
        }
        if (right_edge) {
            hm_r[f] = ld_plain<COH>(fin.rest(f) + row + xp);
            hn_r[f] = SW::to_c(ld_plain<COH>(fin.mov(f, 2) + row + xp));
        }
    }

    // The x part (own outgoing populations, shuffles, halos) and the y part (pulled rows) are
    // independent; their order only changes the compiler's schedule, and the faster order was
    // measured per storage format (FP16: y first, 78.4 against 76.3 GLUPS on the 4096^2 shear
    // layer; BF16: x first, 77.6 against 66.8).  The y part is written out at both places:
    // moved into a function or a lambda, the FP16 order lost its gain (76.2).
    constexpr bool kYFirst = std::is_same<S, __half>::value;
    float2 nown[3][P], B[3][4][P];
    if constexpr (kYFirst) {
#pragma unroll
        for (int q = 0; q < P; ++q) {   // +y from row y - 1, -y from row y + 1
            {
                const float2 ms[3] = {mym[0][q], mym[1][q], mym[2][q]};
                const float2 n[3] = {SW::unpack2(n_py_pull[0][q]), SW::unpack2(n_py_pull[1][q]),
                                     SW::unpack2(n_py_pull[2][q])};
                float2 fl[3], o[3];
                fluxes_d2q5<float2, 1>(k, ms[0], ms[1], ms[2], fl);
                outgoing<float2, 3, +1>(k, ms, fl, n, o);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][2][q] = o[f];
            }
            {
                const float2 ms[3] = {myp[0][q], myp[1][q], myp[2][q]};
                const float2 n[3] = {SW::unpack2(n_my_pull[0][q]), SW::unpack2(n_my_pull[1][q]),
                                     SW::unpack2(n_my_pull[2][q])};
                float2 fl[3], o[3];
                fluxes_d2q5<float2, 1>(k, ms[0], ms[1], ms[2], fl);
                outgoing<float2, 3, -1>(k, ms, fl, n, o);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][3][q] = o[f];
            }
        }
    }
    // ---- own non-equilibrium sum and the outgoing x populations of the lane's own nodes
    float2 ox_p[3][P], ox_m[3][P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        float2 a[3], b[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            a[f] = SW::unpack2(n_px[f][q]);
            b[f] = SW::unpack2(n_mx[f][q]);
            nown[f][q] = p_add(p_add(a[f], b[f]), p_add(SW::unpack2(n_py_own[f][q]), SW::unpack2(n_my_own[f][q])));
        }
        const float2 mq[3] = {mo[0][q], mo[1][q], mo[2][q]};
        float2 fl[3], op[3], om[3];
        fluxes_d2q5<float2, 0>(k, mq[0], mq[1], mq[2], fl);
        outgoing<float2, 3, +1>(k, mq, fl, a, op);
        outgoing<float2, 3, -1>(k, mq, fl, b, om);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            ox_p[f][q] = op[f];
            ox_m[f][q] = om[f];
        }
    }
    // halo nodes x0 - 1 (+x population) and x0 + V (-x population), on the edge lanes only
    float halo_p[3] = {0.0f, 0.0f, 0.0f}, halo_m[3] = {0.0f, 0.0f, 0.0f};
    if (left_edge) {
        float fl[3];
        fluxes_d2q5<float, 0>(k, hm_l[0], hm_l[1], hm_l[2], fl);
        outgoing<float, 3, +1>(k, hm_l, fl, hn_l, halo_p);
    }
    if (right_edge) {
        float fl[3];
        fluxes_d2q5<float, 0>(k, hm_r[0], hm_r[1], hm_r[2], fl);
        outgoing<float, 3, -1>(k, hm_r, fl, hn_r, halo_m);
    }
    // pulled populations B[f][l][q] (l = 0..3 for velocities 1..4): +x from x - 1, -x from x + 1
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const float from_left = __shfl_up_sync(0xffffffffu, ox_p[f][P - 1].y, 1);
        const float from_right = __shfl_down_sync(0xffffffffu, ox_m[f][0].x, 1);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            B[f][0][q] = make_float2(q == 0 ? (left_edge ? halo_p[f] : from_left) : ox_p[f][q - 1].y, ox_p[f][q].x);
            B[f][1][q] = make_float2(ox_m[f][q].y, q == P - 1 ? (right_edge ? halo_m[f] : from_right) : ox_m[f][q + 1].x);
        }
    }
    if constexpr (!kYFirst) {
#pragma unroll
        for (int q = 0; q < P; ++q) {   // +y from row y - 1, -y from row y + 1
            {
                const float2 ms[3] = {mym[0][q], mym[1][q], mym[2][q]};
                const float2 n[3] = {SW::unpack2(n_py_pull[0][q]), SW::unpack2(n_py_pull[1][q]),
                                     SW::unpack2(n_py_pull[2][q])};
                float2 fl[3], o[3];
                fluxes_d2q5<float2, 1>(k, ms[0], ms[1], ms[2], fl);
                outgoing<float2, 3, +1>(k, ms, fl, n, o);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][2][q] = o[f];
            }
            {
                const float2 ms[3] = {myp[0][q], myp[1][q], myp[2][q]};
                const float2 n[3] = {SW::unpack2(n_my_pull[0][q]), SW::unpack2(n_my_pull[1][q]),
                                     SW::unpack2(n_my_pull[2][q])};
                float2 fl[3], o[3];
                fluxes_d2q5<float2, 1>(k, ms[0], ms[1], ms[2], fl);
                outgoing<float2, 3, -1>(k, ms, fl, n, o);
#pragma unroll
                for (int f = 0; f < 3; ++f) B[f][3][q] = o[f];
            }
        }
    }

    // ---- new moments, their equilibrium, relaxed non-equilibrium parts
    //   m' = m + (sum_l B_l - 4 alpha_s m - sum_l n_l) / s
    //   n'_l = (1 - omega) (B_l - alpha_s m' -+ flux_l(m'))
    uint32_t out_n[3][4][P];
    float2 out_m[3][P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        float2 m[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const float2 pulled = p_add(p_add(B[f][0][q], B[f][1][q]), p_add(B[f][2][q], B[f][3][q]));
            const float2 d = p_sub(p_fma(k.p_nal4[f], mo[f][q], pulled), nown[f][q]);
            m[f] = p_fma(k.p_inv_s, d, mo[f][q]);
        }
        float2 fx[3], fy[3];
        fluxes_d2q5_xy<float2>(k, m[0], m[1], m[2], fx, fy);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const float2 base = p_mul(k.p_nwal[f], m[f]);     // -(1 - omega) alpha_s m'
            const float2 w = k.p_w[f];
            out_n[f][0][q] = SW::pack2(p_fma(w, p_sub(B[f][0][q], fx[f]), base));
            out_n[f][1][q] = SW::pack2(p_fma(w, p_add(B[f][1][q], fx[f]), base));
            out_n[f][2][q] = SW::pack2(p_fma(w, p_sub(B[f][2][q], fy[f]), base));
            out_n[f][3][q] = SW::pack2(p_fma(w, p_add(B[f][3][q], fy[f]), base));
            out_m[f][q] = m[f];
        }
        if constexpr (DIAG) {
            if (active) accumulate_pair(acc, m[0], &m[1], 2, k.rho_bar);
        }
    }
    if (active) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            float wm[V];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                wm[2 * q] = out_m[f][q].x;
                wm[2 * q + 1] = out_m[f][q].y;
            }
            vstore<float, V>(fout.rest(f) + row + x0, wm);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                W w;
                memcpy(&w, &out_n[f][l][0], sizeof(W));
                *reinterpret_cast<W*>(fout.mov(f, l + 1) + row + x0) = w;
            }
        }
    }
}

// At least two resident blocks per SM (at most 128 registers): the BF16 instantiation with
// fused diagnostics needs 131 and would otherwise run one block per SM.  The two-node-per-lane
// plain step fits 80 registers and runs three blocks per SM (71.2 against 59.0 GLUPS at two).
template <class S, int V, bool DIAG>
__global__ void __launch_bounds__(kThreads, (V == 2 && !DIAG) ? 3 : 2)
k_split_step_2d_vec(const char* __restrict__ fin_b, char* __restrict__ fout_b, int nx, int ny, long long plane,
                    FastDiv wdiv, Coef<typename Storage<S>::C> k, DiagSink sink,
                    uint32_t* __restrict__ step_ctr, int par) {
    using L = Layout<S, true, 5>;
    const L fin{const_cast<char*>(fin_b), plane}, fout{fout_b, plane};
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    take_step_key(step_ctr, par);   // keeps the step counter in step (the split forms round to nearest)
    AccPair acc;
    if (DIAG) acc.zero();
    const uint32_t items = (uint32_t)ny * wdiv.d;
    for (uint32_t item = gwarp; item < items; item += (DIAG ? nwarps : items)) {   // warp-uniform
        const uint32_t y = wdiv.div(item);
        warp_split_step_2d<S, V, DIAG>(fin, fout, nx, ny, (int)y, (int)(item - y * wdiv.d), lane, k, acc);
    }
    if (DIAG) {
        Acc<float> a = acc.fold();
        block_reduce_finish(a, sink);
    }
}

// One node of the 2D split step (the per-node kernel's body; also the batched step's path for
// problems whose n_x is not a multiple of its vector width).  COH: coherent loads.
template <class S, bool DIAG, bool COH = false>
__device__ __forceinline__ void node_split_step_2d(const Layout<S, true, 5>& fin, const Layout<S, true, 5>& fout,
                                                   int nx, int ny, long long node, const Coef<float>& k,
                                                   Acc<float>& acc) {
    using C = float;
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
    for (int f = 0; f < 3; ++f) m[f] = ld_plain<COH>(fin.rest(f) + node);
#pragma unroll
    for (int l = 1; l < 5; ++l) {
        C ms[3], np[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            ms[f] = ld_plain<COH>(fin.rest(f) + src[l]);
            np[f] = Storage<S>::to_c(ld_plain<COH>(fin.mov(f, l) + src[l]));      // stored units
            nown[f] += Storage<S>::to_c(ld_plain<COH>(fin.mov(f, l) + node));
        }
        if (l == 1) pulled_d2q5<C, 1>(k, ms, np, B);
        else if (l == 2) pulled_d2q5<C, 2>(k, ms, np, B);
        else if (l == 3) pulled_d2q5<C, 3>(k, ms, np, B);
        else pulled_d2q5<C, 4>(k, ms, np, B);
    }
    split_update_d2q5(k, m, B, nown);
    if constexpr (DIAG) {
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
         node += (DIAG ? (long long)gridDim.x * blockDim.x : plane))
        node_split_step_2d<S, DIAG>(fin, fout, nx, ny, node, k, acc);
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

// One row segment of the 3D split step: two nodes per lane (one pair) along x; sources x -+ 1
// by warp shuffle of the lane's outgoing x populations (the edge lanes evaluate the halo
// node's population themselves), y -+ 1 rows and z -+ 1 planes.
template <class S, bool DIAG, class In, class Out, class A>
__device__ __forceinline__ void warp_split_step_3d(const In& fin, const Out& fout, int nx, int ny, int nz, int y, int z,
                                                   int seg, int lane, const Coef<float>& k, A& acc) {
    static_assert(kSplitV3 == 2, "one node pair per lane");
    using SW = Storage<S>;
    const int x0 = (seg * 32 + lane) * 2;
    const bool active = x0 < nx;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const uint32_t unx = nx, uny = ny;
    const uint32_t row = ((uint32_t)z * uny + y) * unx;
    const uint32_t src_row[4] = {((uint32_t)z * uny + ym) * unx, ((uint32_t)z * uny + yp) * unx,
                                 ((uint32_t)zm * uny + y) * unx, ((uint32_t)zp * uny + y) * unx};
    const uint32_t xm = x0 == 0 ? nx - 1 : x0 - 1;
    const uint32_t xp = x0 + 2 >= nx ? 0 : x0 + 2;
    const uint32_t ux0 = (uint32_t)x0;
    const bool left_edge = lane == 0 && active;
    const bool right_edge = active && (lane == 31 || x0 + 2 >= nx);
    auto ldm = [&](const float* p) {
        return active ? __ldg(reinterpret_cast<const float2*>(p)) : make_float2(0.0f, 0.0f);
    };
    auto ldn = [&](const S* p) { return active ? __ldg(reinterpret_cast<const unsigned int*>(p)) : 0u; };

    // ---- load phase: every load of the lane is issued before the arithmetic (the node pair's
    // moments and six own non-equilibrium parts, the y / z neighbours' moments and pulled parts,
    // the warp-edge halo values)
    float2 m[4], ms[4][4];
    uint32_t wn[4][6], wpull[4][4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        m[f] = ldm(fin.rest(f) + row + ux0);
#pragma unroll
        for (int l = 1; l < 7; ++l) wn[f][l - 1] = ldn(fin.mov(f, l) + row + ux0);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            ms[d][f] = ldm(fin.rest(f) + src_row[d] + ux0);
            wpull[d][f] = ldn(fin.mov(f, 3 + d) + src_row[d] + ux0);
        }
    float hmom_l[4], hn_l[4], hmom_r[4], hn_r[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) hmom_l[f] = hn_l[f] = hmom_r[f] = hn_r[f] = 0.0f;
    if (left_edge) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            hmom_l[f] = fin.rest(f)[row + xm];
            hn_l[f] = SW::to_c(fin.mov(f, 1)[row + xm]);
        }
    }
    if (right_edge) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            hmom_r[f] = fin.rest(f)[row + xp];
            hn_r[f] = SW::to_c(fin.mov(f, 2)[row + xp]);
        }
    }

    // ---- outgoing +x / -x populations of the lane's own nodes, shifted by one node
    float2 nown[4], B[4][6];
    {
        float2 a[4], b[4], fl[4], op[4], om[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            a[f] = SW::unpack2(wn[f][0]);
            b[f] = SW::unpack2(wn[f][1]);
            nown[f] = p_add(p_add(a[f], b[f]), p_add(p_add(SW::unpack2(wn[f][2]), SW::unpack2(wn[f][3])),
                                                     p_add(SW::unpack2(wn[f][4]), SW::unpack2(wn[f][5]))));
        }
        fluxes_d3q7<float2, 0>(k, m, fl);
        outgoing<float2, 4, +1>(k, m, fl, a, op);
        outgoing<float2, 4, -1>(k, m, fl, b, om);
        float hp[4] = {0.0f, 0.0f, 0.0f, 0.0f}, hm[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (left_edge) {
            float hfl[4];
            fluxes_d3q7<float, 0>(k, hmom_l, hfl);
            outgoing<float, 4, +1>(k, hmom_l, hfl, hn_l, hp);
        }
        if (right_edge) {
            float hfl[4];
            fluxes_d3q7<float, 0>(k, hmom_r, hfl);
            outgoing<float, 4, -1>(k, hmom_r, hfl, hn_r, hm);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float from_left = __shfl_up_sync(0xffffffffu, op[f].y, 1);
            const float from_right = __shfl_down_sync(0xffffffffu, om[f].x, 1);
            B[f][0] = make_float2(left_edge ? hp[f] : from_left, op[f].x);
            B[f][1] = make_float2(om[f].y, right_edge ? hm[f] : from_right);
        }
    }
    // +y, -y, +z, -z from rows y -+ 1 and planes z -+ 1
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int l = 3 + d;
        float2 n[4], fl[4], o[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) n[f] = SW::unpack2(wpull[d][f]);
        if (d < 2) fluxes_d3q7<float2, 1>(k, ms[d], fl);
        else fluxes_d3q7<float2, 2>(k, ms[d], fl);
        if (d % 2 == 0) outgoing<float2, 4, +1>(k, ms[d], fl, n, o);
        else outgoing<float2, 4, -1>(k, ms[d], fl, n, o);
#pragma unroll
        for (int f = 0; f < 4; ++f) B[f][l - 1] = o[f];
    }

    // new moments m' = m + (sum_l B_l - 6 alpha_s m - sum_l n_l) / s (6 alpha_s m as 6 (alpha_s m),
    // the moving equilibria's exact sum), their fluxes, relaxed parts (1 - omega)(B_l - e_l(m'))
    const float2 six = make_float2(-6.0f, -6.0f);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float2 pulled = p_add(p_add(p_add(B[f][0], B[f][1]), p_add(B[f][2], B[f][3])), p_add(B[f][4], B[f][5]));
        const float2 d = p_sub(p_fma(six, p_mul(k.p_al[f], m[f]), pulled), nown[f]);
        m[f] = p_fma(k.p_inv_s, d, m[f]);
    }
    float2 fl[3][4];
    fluxes_d3q7_all<float2>(k, m, fl);
    if constexpr (DIAG) {
        if (active) accumulate_pair(acc, m[0], &m[1], 3, k.rho_bar);
    }
    if (active) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            *reinterpret_cast<float2*>(fout.rest(f) + row + ux0) = m[f];
            const float2 base = p_mul(k.p_nwal[f], m[f]);     // -(1 - omega) alpha_s m'
            const float2 w = k.p_w[f];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const uint32_t up = SW::pack2(p_fma(w, p_sub(B[f][2 * a], fl[a][f]), base));
                const uint32_t dn = SW::pack2(p_fma(w, p_add(B[f][2 * a + 1], fl[a][f]), base));
                *reinterpret_cast<unsigned int*>(fout.mov(f, 2 * a + 1) + row + ux0) = up;
                *reinterpret_cast<unsigned int*>(fout.mov(f, 2 * a + 2) + row + ux0) = dn;
            }
        }
    }
}

// Two resident blocks per SM (at most 128 registers): the 24 pulled populations of a node
// pair stay live until the new moments are known, and below 128 registers the compiler
// spills them and recomputes plane addresses.
template <class S, bool DIAG>
__global__ void __launch_bounds__(kThreads, 2)
k_split_step_3d_vec(const SplitPlanes<S, 7> P, int nx, int ny, int nz, FastDiv wdiv, FastDiv ydiv,
                    Coef<typename Storage<S>::C> k, DiagSink sink, uint32_t* __restrict__ step_ctr, int par) {
    const PlanesIn<S, 7> fin{P};
    const PlanesOut<S, 7> fout{P};
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    take_step_key(step_ctr, par);   // keeps the step counter in step (the split forms round to nearest)
    AccPair acc;
    if (DIAG) acc.zero();
    const uint32_t items = (uint32_t)ny * (uint32_t)nz * wdiv.d;
    for (uint32_t item = gwarp; item < items; item += (DIAG ? nwarps : items)) {   // warp-uniform
        const uint32_t r = wdiv.div(item);
        const uint32_t z = ydiv.div(r);
        warp_split_step_3d<S, DIAG>(fin, fout, nx, ny, nz, (int)(r - z * (uint32_t)ny), (int)z,
                                    (int)(item - r * wdiv.d), lane, k, acc);
    }
    if (DIAG) {
        Acc<float> a = acc.fold();
        block_reduce_finish(a, sink);
    }
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
