/*
 * FP64 CPU oracle of the vectorial lattice Boltzmann scheme
 * (Aregba-Driollet, Bellotti, Natalini, Tenna, Section 2, Eq. LBM_scheme).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the package smoke check
 * and the benchmark's CPU-baseline leg; never by the product path.  Shares no
 * code with the CUDA path.  Built with -O2 -ffp-contract=off so that every
 * operation is the rounded FP64 operation written here.
 *
 * Each routine states the passage of the paper it follows.  Where the paper is
 * garbled or silent the reading taken is written beside the code:
 *   (R1) the rest equilibrium of a momentum field carries the factor dx,
 *        dx (1 - 4 alpha_q) q, because the moment of that field is
 *        sum_l f_l = dx q (Section 2) and the proof of Prop. 1 uses the row
 *        (1/dx, ..., 1/dx) for q and s^eq = 2 dx alpha q;
 *   (R2) transport is periodic: node index i +- 1 taken modulo n;
 *   (R3) summation order of moments is l = 0, 1, 2, 3, 4 (, 5, 6);
 *   (R4) 3D (D3Q7) equilibria follow the 2D ones direction by direction
 *        (the paper only states that the extension is straightforward):
 *        rest (1 - 6 alpha) rho / dx (1 - 6 alpha_j) q_j; direction +-e_d:
 *        alpha rho +- dx/(2 mu) q_d and
 *        dx alpha_j q_j +- dx^2/(2 mu) q_j q_d / rho +- delta_jd P(rho)/(2 mu).
 */
#include "vlbm_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXQ 7
#define MAXF 4
#define MAXP (MAXQ * MAXF)

int orc_q(const orc_params* p) { return p->dim == 3 ? 7 : 5; }
int orc_fields(const orc_params* p) { return p->dim + 1; }
long orc_nodes(const orc_params* p) { return p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1); }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops (timing only: the step has no reductions, so the
 * result does not depend on the thread count). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Pressure law P(rho) = rho^gamma, gamma >= 1 (Section 2, footnote). */
static double pressure(const orc_params* p, double rho) { return pow(rho, p->gamma); }

/* Equilibria of the D2Q5 vectorial scheme, written entry by entry as printed
 * in Section 2 (velocities 0, +x, -x, +y, -y; fields rho, q_x, q_y). */
static void equilibrium_d2q5(const orc_params* p, double rho, double qx, double qy, double* feq)
{
    const double dx = p->dx, mu = p->mu;
    const double ar = p->alpha[0], ax = p->alpha[1], ay = p->alpha[2];
    const double P = pressure(p, rho);
    double* fr = feq;        /* field rho */
    double* fx = feq + 5;    /* field q_x */
    double* fy = feq + 10;   /* field q_y */

    /* rest velocity */
    fr[0] = (1.0 - 4.0 * ar) * rho;
    fx[0] = dx * (1.0 - 4.0 * ax) * qx;   /* (R1) */
    fy[0] = dx * (1.0 - 4.0 * ay) * qy;   /* (R1) */

    /* +x */
    fr[1] = ar * rho + dx / (2.0 * mu) * qx;
    fx[1] = dx * ax * qx + dx * dx / (2.0 * mu) * qx * qx / rho + P / (2.0 * mu);
    fy[1] = dx * ay * qy + dx * dx / (2.0 * mu) * qx * qy / rho;

    /* -x */
    fr[2] = ar * rho - dx / (2.0 * mu) * qx;
    fx[2] = dx * ax * qx - dx * dx / (2.0 * mu) * qx * qx / rho - P / (2.0 * mu);
    fy[2] = dx * ay * qy - dx * dx / (2.0 * mu) * qx * qy / rho;

    /* +y */
    fr[3] = ar * rho + dx / (2.0 * mu) * qy;
    fx[3] = dx * ax * qx + dx * dx / (2.0 * mu) * qx * qy / rho;
    fy[3] = dx * ay * qy + dx * dx / (2.0 * mu) * qy * qy / rho + P / (2.0 * mu);

    /* -y */
    fr[4] = ar * rho - dx / (2.0 * mu) * qy;
    fx[4] = dx * ax * qx - dx * dx / (2.0 * mu) * qx * qy / rho;
    fy[4] = dx * ay * qy - dx * dx / (2.0 * mu) * qy * qy / rho - P / (2.0 * mu);
}

/* D3Q7 equilibria, reading (R4). Velocity 2d+1 is +e_d, 2d+2 is -e_d. */
static void equilibrium_d3q7(const orc_params* p, double rho, const double* q, double* feq)
{
    const double dx = p->dx, mu = p->mu;
    const double P = pressure(p, rho);
    /* field rho */
    feq[0] = (1.0 - 6.0 * p->alpha[0]) * rho;
    for (int d = 0; d < 3; ++d) {
        feq[1 + 2 * d] = p->alpha[0] * rho + dx / (2.0 * mu) * q[d];
        feq[2 + 2 * d] = p->alpha[0] * rho - dx / (2.0 * mu) * q[d];
    }
    /* field q_j */
    for (int j = 0; j < 3; ++j) {
        double* fj = feq + 7 * (j + 1);
        const double aj = p->alpha[j + 1];
        fj[0] = dx * (1.0 - 6.0 * aj) * q[j];
        for (int d = 0; d < 3; ++d) {
            const double flux = dx * dx / (2.0 * mu) * q[j] * q[d] / rho + (j == d ? P / (2.0 * mu) : 0.0);
            fj[1 + 2 * d] = dx * aj * q[j] + flux;
            fj[2 + 2 * d] = dx * aj * q[j] - flux;
        }
    }
}

void orc_equilibrium(const orc_params* p, double rho, const double* q, double* feq)
{
    if (p->dim == 3)
        equilibrium_d3q7(p, rho, q, feq);
    else
        equilibrium_d2q5(p, rho, q[0], q[1], feq);
}

/* Conserved moments of one node (Section 2): rho = sum_l f^rho_l,
 * dx q_d = sum_l f^{q_d}_l, summed in the order l = 0, 1, ... (R3). */
static void node_moments(const orc_params* p, const double* f, double* rho, double* q)
{
    const int Q = orc_q(p);
    double s = 0.0;
    for (int l = 0; l < Q; ++l) s += f[l];
    *rho = s;
    for (int d = 0; d < p->dim; ++d) {
        double t = 0.0;
        for (int l = 0; l < Q; ++l) t += f[(d + 1) * Q + l];
        q[d] = t / p->dx;
    }
}

/* Relaxation as in Eq. LBM_scheme: f* = (1 - omega_k) f + omega_k f^eq,
 * field by field. */
static void collide_populations(const orc_params* p, const double* f, double* out)
{
    const int Q = orc_q(p), F = orc_fields(p);
    double rho, q[3] = {0.0, 0.0, 0.0}, feq[MAXP];
    node_moments(p, f, &rho, q);
    orc_equilibrium(p, rho, q, feq);
    for (int k = 0; k < F; ++k)
        for (int l = 0; l < Q; ++l)
            out[k * Q + l] = (1.0 - p->omega[k]) * f[k * Q + l] + p->omega[k] * feq[k * Q + l];
}

/* Relaxation written on moments, as in the proof of Prop. 1: for each field
 * the moments are the conserved one m (sum of the populations, divided by dx
 * for a momentum field), and per direction d the antisymmetric
 * a_d = f_{+d} - f_{-d} and symmetric s_d = f_{+d} + f_{-d} ones.  m is kept,
 * a_d and s_d relax toward their equilibrium values, then the populations are
 * rebuilt: f_{+d} = (s_d + a_d)/2, f_{-d} = (s_d - a_d)/2,
 * f_0 = (dx) m - sum_d s_d.  The equilibrium moments are those of the proof:
 *   field q_j: a_d^eq = dx^2/mu q_j q_d / rho + delta_jd P/mu, s_d^eq = 2 dx alpha_j q_j;
 *   field rho: a_d^eq = dx/mu q_d,                          s_d^eq = 2 alpha_rho rho. */
static void collide_moments(const orc_params* p, const double* f, double* out)
{
    const int Q = orc_q(p), F = orc_fields(p), D = p->dim;
    const double dx = p->dx, mu = p->mu;
    double rho, q[3] = {0.0, 0.0, 0.0};
    node_moments(p, f, &rho, q);
    const double P = pressure(p, rho);
    for (int k = 0; k < F; ++k) {
        const double* fk = f + k * Q;
        double* ok = out + k * Q;
        const double w = p->omega[k];
        const double m = (k == 0) ? rho : dx * q[k - 1];   /* population sum of field k */
        double ssum = 0.0;
        for (int d = 0; d < D; ++d) {
            const double a = fk[1 + 2 * d] - fk[2 + 2 * d];
            const double s = fk[1 + 2 * d] + fk[2 + 2 * d];
            double a_eq, s_eq;
            if (k == 0) {
                a_eq = dx / mu * q[d];
                s_eq = 2.0 * p->alpha[0] * rho;
            } else {
                const int j = k - 1;
                a_eq = dx * dx / mu * q[j] * q[d] / rho + (j == d ? P / mu : 0.0);
                s_eq = 2.0 * dx * p->alpha[k] * q[j];
            }
            const double a_s = (1.0 - w) * a + w * a_eq;
            const double s_s = (1.0 - w) * s + w * s_eq;
            ok[1 + 2 * d] = 0.5 * (s_s + a_s);
            ok[2 + 2 * d] = 0.5 * (s_s - a_s);
            ssum += s_s;
        }
        ok[0] = m - ssum;
    }
}

static void collide_node(const orc_params* p, const double* f, double* out, int form)
{
    if (form == ORC_COLLIDE_MOMENTS)
        collide_moments(p, f, out);
    else
        collide_populations(p, f, out);
}

void orc_collide_nodes(const orc_params* p, long count, const double* f, double* out, int form)
{
    const int P = orc_fields(p) * orc_q(p);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < count; ++i) collide_node(p, f + i * P, out + i * P, form);
}

void orc_collide_lattice(const orc_params* p, const double* f, double* out, int form)
{
    const int P = orc_fields(p) * orc_q(p);
    const long N = orc_nodes(p);
    const long nrows = N / p->n[0];
#pragma omp parallel for schedule(static)
    for (long row = 0; row < nrows; ++row) {
        double fn[MAXP], on[MAXP];
        for (long x = 0; x < p->n[0]; ++x) {
            const long node = row * p->n[0] + x;
            for (int c = 0; c < P; ++c) fn[c] = f[c * N + node];
            collide_node(p, fn, on, form);
            for (int c = 0; c < P; ++c) out[c * N + node] = on[c];
        }
    }
}

/* Transport (Section 2): f_l(t + dt, x) = f*_l(t, x - c_l dx), with periodic
 * wrap (R2).  Velocity 2d+1 moves along +e_d, 2d+2 along -e_d. */
void orc_stream(const orc_params* p, const double* fs, double* f)
{
    const int Q = orc_q(p), F = orc_fields(p);
    const long nx = p->n[0], ny = p->n[1], nz = (p->dim == 3 ? p->n[2] : 1);
    const long N = nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < nz; ++z) {
        for (long y = 0; y < ny; ++y) {
            for (long x = 0; x < nx; ++x) {
                const long node = (z * ny + y) * nx + x;
                for (int k = 0; k < F; ++k) {
                    for (int l = 0; l < Q; ++l) {
                        long sx = x, sy = y, sz = z;   /* source node x - c_l */
                        switch (l) {
                            case 1: sx = (x - 1 + nx) % nx; break;
                            case 2: sx = (x + 1) % nx; break;
                            case 3: sy = (y - 1 + ny) % ny; break;
                            case 4: sy = (y + 1) % ny; break;
                            case 5: sz = (z - 1 + nz) % nz; break;
                            case 6: sz = (z + 1) % nz; break;
                            default: break;
                        }
                        const long src = (sz * ny + sy) * nx + sx;
                        const long plane = (long)(k * Q + l) * N;
                        f[plane + node] = fs[plane + src];
                    }
                }
            }
        }
    }
}

void orc_run(const orc_params* p, double* f, double* work, long nsteps, int form)
{
    for (long s = 0; s < nsteps; ++s) {
        orc_collide_lattice(p, f, work, form);
        orc_stream(p, work, f);
    }
}

/* Initialisation at equilibrium (end of Section 2), with the density taken
 * from the pressure expansion of Prop. 1: P(rho) = P(rho_bar) + dx^2 rho_bar phi,
 * and q = rho u. */
void orc_init(const orc_params* p, const double* u, const double* phi, double* f)
{
    const int P = orc_fields(p) * orc_q(p);
    const long N = orc_nodes(p);
#pragma omp parallel for schedule(static)
    for (long node = 0; node < N; ++node) {
        const double ph = phi ? phi[node] : 0.0;
        const double rho = pow(pressure(p, p->rho_bar) + p->dx * p->dx * p->rho_bar * ph, 1.0 / p->gamma);
        double q[3] = {0.0, 0.0, 0.0}, feq[MAXP];
        for (int d = 0; d < p->dim; ++d) q[d] = rho * u[d * N + node];
        orc_equilibrium(p, rho, q, feq);
        for (int c = 0; c < P; ++c) f[c * N + node] = feq[c];
    }
}

void orc_macros(const orc_params* p, const double* f, double* rho_out, double* u_out, double* phi_out)
{
    const int P = orc_fields(p) * orc_q(p);
    const long N = orc_nodes(p);
#pragma omp parallel for schedule(static)
    for (long node = 0; node < N; ++node) {
        double fn[MAXP], rho, q[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < P; ++c) fn[c] = f[c * N + node];
        node_moments(p, fn, &rho, q);
        if (rho_out) rho_out[node] = rho;
        if (u_out)
            for (int d = 0; d < p->dim; ++d) u_out[d * N + node] = q[d] / rho;
        if (phi_out)
            phi_out[node] = (pressure(p, rho) - pressure(p, p->rho_bar)) / (p->dx * p->dx * p->rho_bar);
    }
}

void orc_invariants(const orc_params* p, const double* f, double* out)
{
    const int P = orc_fields(p) * orc_q(p);
    const long N = orc_nodes(p);
    double vol = 1.0;
    for (int d = 0; d < p->dim; ++d) vol *= p->dx;
    double srho = 0.0, sq[3] = {0.0, 0.0, 0.0}, ekin = 0.0, umax = 0.0, nonfinite = 0.0, sdev = 0.0;
    for (long node = 0; node < N; ++node) {
        double fn[MAXP], rho, q[3] = {0.0, 0.0, 0.0};
        int bad = 0;
        for (int c = 0; c < P; ++c) {
            fn[c] = f[c * N + node];
            if (!isfinite(fn[c])) bad = 1;
        }
        if (bad) {
            nonfinite += 1.0;
            continue;
        }
        node_moments(p, fn, &rho, q);
        srho += rho;
        sdev += rho - p->rho_bar;
        double q2 = 0.0;
        for (int d = 0; d < p->dim; ++d) {
            sq[d] += q[d];
            q2 += q[d] * q[d];
        }
        ekin += 0.5 * q2 / rho * vol;
        const double speed = sqrt(q2) / rho;
        if (speed > umax) umax = speed;
    }
    out[0] = srho;
    out[1] = sq[0];
    out[2] = sq[1];
    out[3] = sq[2];
    out[4] = ekin;
    out[5] = umax;
    out[6] = nonfinite;
    out[7] = sdev;
}
