/*
 * FP64 CPU oracle of the vectorial lattice Boltzmann scheme
 * (Aregba-Driollet, Bellotti, Natalini, Tenna, Section 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * call or execute this code: only the test-suite, the smoke check of the
 * package entry and the CPU-baseline leg of the benchmark use it.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Lattice layout (plain, no padding):
 *   f[((k * Q + l) * nz + z) * ny + y) * nx + x]
 * with field k = 0 (rho), 1 (q_x), 2 (q_y), 3 (q_z, 3D only) and velocity
 *   2D (D2Q5): l = 0 rest, 1 +x, 2 -x, 3 +y, 4 -y
 *   3D (D3Q7): l = 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z
 * Q = 5 (2D) or 7 (3D); nz = 1 in 2D.  The state f holds the populations
 * BEFORE relaxation at time t = step * dx^2 / mu (Eq. parabolicScaling).
 * Macroscopic arrays: rho/phi (nz, ny, nx), u (d, nz, ny, nx).
 */
#ifndef VLBM_ORACLE_H
#define VLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int    dim;        /* 2 or 3 */
    long   n[3];       /* nx, ny, nz (nz = 1 in 2D); periodic */
    double dx;         /* space step */
    double mu;         /* parabolic scaling dx^2 / dt */
    double gamma;      /* pressure law P(rho) = rho^gamma */
    double rho_bar;    /* reference density */
    double omega[4];   /* relaxation parameter of field k */
    double alpha[4];   /* linear-equilibrium coefficient of field k */
} orc_params;

enum { ORC_COLLIDE_POPULATIONS = 0, ORC_COLLIDE_MOMENTS = 1 };

int  orc_q(const orc_params* p);        /* velocities per field */
int  orc_fields(const orc_params* p);   /* dim + 1 */
long orc_nodes(const orc_params* p);
int  orc_num_threads(void);
void orc_set_num_threads(int n);

/* Equilibrium of one node: feq[k * Q + l]. */
void orc_equilibrium(const orc_params* p, double rho, const double* q, double* feq);

/* Relaxation of `count` nodes stored node-major: f[node * (fields*Q) + k*Q + l]. */
void orc_collide_nodes(const orc_params* p, long count, const double* f, double* out, int form);

/* Relaxation of the whole lattice (lattice layout) into out. */
void orc_collide_lattice(const orc_params* p, const double* f, double* out, int form);

/* Transport of post-relaxation populations fs into f (periodic). */
void orc_stream(const orc_params* p, const double* fs, double* f);

/* nsteps of relax-then-transport; work has the size of f. */
void orc_run(const orc_params* p, double* f, double* work, long nsteps, int form);

/* Initialisation at equilibrium from u (and phi, may be NULL). */
void orc_init(const orc_params* p, const double* u, const double* phi, double* f);

/* Macroscopic fields; any output may be NULL. */
void orc_macros(const orc_params* p, const double* f, double* rho, double* u, double* phi);

/* out[8] = { sum rho, sum q_x, sum q_y, sum q_z, E_kin, max|u|, non-finite nodes,
 *            sum (rho - rho_bar) },  E_kin = 1/2 sum |q|^2 / rho * dx^d. */
void orc_invariants(const orc_params* p, const double* f, double* out);

#ifdef __cplusplus
}
#endif
#endif
