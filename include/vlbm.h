/*
 * vlbm — C ABI of the B300 (sm_103a) implementation of the vectorial lattice
 * Boltzmann scheme for incompressible Navier-Stokes (Aregba-Driollet,
 * Bellotti, Natalini, Tenna): each conserved field (rho, q_x, q_y[, q_z])
 * carries its own D2Q5 (3D: D3Q7) population set, relaxes toward its own
 * equilibrium (Section 2, Eq. LBM_scheme) under the parabolic scaling
 * dx^2 / dt = mu (Eq. parabolicScaling), then streams on a periodic
 * Cartesian lattice with nodes at half-integer positions (i + 1/2) dx.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: VLBM_OK (0) on success, a positive warning code, or a
 *    negative error code (VLBM_E*).  No exception crosses the ABI; no global
 *    state; a handle is not thread-safe (one host thread at a time).
 *  - Caller arrays are contiguous, x fastest: scalar fields (rho, phi) are
 *    [ny][nx] (3D: [nz][ny][nx]); vector fields (u) are [d][ny][nx]
 *    (3D: [d][nz][ny][nx]).  Their element type is given by a VLBM_DTYPE_*.
 *  - Pointers may be device memory or host memory (pinned or pageable): the
 *    library asks the CUDA driver which one it is.  Host arrays are staged
 *    through a device buffer that the handle owns, and a call that reads
 *    back into host memory synchronises the handle's stream before it
 *    returns.  Device arrays are used in place, in stream order.
 *  - All GPU work of a handle is enqueued on the stream given at creation
 *    (or by vlbm_set_stream); NULL means the legacy default stream.
 *  - The handle owns its population lattices and scratch buffers; the caller
 *    owns every array it passes.  Nothing is retained after a call returns.
 *  - The populations held by a handle are the post-relaxation values f*(t);
 *    their moments equal those of f(t) because relaxation conserves them.
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define VLBM_OK            0
#define VLBM_WSTABILITY    1   /* created; mu is below the low-frequency stability bound (Lemma 2) */
#define VLBM_EINVAL       -1   /* null pointer, bad size, parameter outside its range */
#define VLBM_ESTABILITY   -2   /* strict mode: mu below the low-frequency bound (Lemma 2) */
#define VLBM_ENOMEM       -3   /* device or host allocation failed */
#define VLBM_ECUDA        -4   /* a CUDA call failed; vlbm_last_error() has the message */
#define VLBM_EDIVERGED    -5   /* a non-finite population was found (check requested) */
#define VLBM_ETIMEOUT     -6   /* a bounded device wait gave up */
#define VLBM_EUNSUPPORTED -7   /* valid request this build does not implement */

/* ---- population storage ------------------------------------------------ */
#define VLBM_FP64          0   /* FP64 storage of deviations from the rest equilibrium, FP64 arithmetic */
#define VLBM_FP32          1   /* FP32 storage of deviations from the rest equilibrium, FP32 arithmetic */
#define VLBM_FP16_SHIFTED  2   /* FP16 storage of scaled deviations, FP32 arithmetic */
#define VLBM_BF16_SHIFTED  3   /* BF16 storage of scaled deviations, FP32 arithmetic */
#define VLBM_FP16_SPLIT    4   /* rest populations FP32, moving populations FP16 (scaled deviations), FP32 arithmetic */
#define VLBM_BF16_SPLIT    5   /* rest populations FP32, moving populations BF16 (scaled deviations), FP32 arithmetic */

/* ---- element type of caller arrays ------------------------------------- */
#define VLBM_DTYPE_F32     0
#define VLBM_DTYPE_F64     1

/* ---- vlbm_step flags ---------------------------------------------------- */
#define VLBM_STEP_CHECK_FINITE 1  /* after stepping, scan the lattice; VLBM_EDIVERGED if non-finite */
#define VLBM_STEP_NO_GRAPH     2  /* launch kernel by kernel instead of replaying a captured CUDA graph */
#define VLBM_STEP_PERSISTENT   4  /* vlbm_batch_step only: all steps in one cooperative launch (below) */
#define VLBM_STEP_TEST_TIMEOUT 8  /* with VLBM_STEP_PERSISTENT: test of the timeout path (below) */

/* Number of doubles written by vlbm_invariants. */
#define VLBM_NUM_INVARIANTS 8

typedef struct vlbm_handle vlbm_handle;

/* Scheme parameters (Section 2).  Field index k: 0 = rho, 1 = q_x, 2 = q_y, 3 = q_z. */
typedef struct {
    int32_t dim;         /* 2 (D2Q5, 3 fields x 5 velocities) or 3 (D3Q7, 4 fields x 7) */
    int32_t precision;   /* VLBM_FP64 | VLBM_FP32 | VLBM_FP16_SHIFTED | VLBM_BF16_SHIFTED |
                            VLBM_FP16_SPLIT | VLBM_BF16_SPLIT */
    int64_t n[3];        /* nodes along x, y, z (n[2] ignored in 2D); each >= 1; periodic */
    double  dx;          /* space step > 0; the periodic box is n[d] * dx long */
    double  mu;          /* parabolic scaling dx^2 / dt > 0 (Eq. parabolicScaling) */
    double  nu;          /* target viscosity >= 0, used for every momentum field with alpha[k] < 0 */
    double  omega[4];    /* relaxation parameter of field k, in (0, 2) (2 is inviscid, Prop. 1) */
    double  alpha[4];    /* linear-equilibrium coefficient of field k, in [0, 1/4] (2D, Lemma 1)
                            or [0, 1/6] (3D); a momentum field with alpha < 0 takes
                            alpha = nu / (2 mu (1/omega - 1/2)) (Prop. 1) */
    double  gamma;       /* pressure law P(rho) = rho^gamma, gamma >= 1 (Section 2) */
    double  rho_bar;     /* reference density > 0 (rest state, Prop. 1) */
    int32_t strict;      /* nonzero: a mu below the Lemma 2 bound is VLBM_ESTABILITY, not a warning */
    int32_t reserved;    /* must be 0 */
} vlbm_params;

/* Quantities derived from vlbm_params by vlbm_params_check. */
typedef struct {
    double  dt;                   /* dx^2 / mu */
    double  alpha[4];             /* resolved alpha per field */
    double  viscosity[4];         /* 2 mu alpha_k (1/omega_k - 1/2), the diffusion of field k (Prop. 1) */
    double  mu_min;               /* (alpha_rho + min_k alpha_qk)^(-1/2): low-frequency acoustic bound */
    int64_t nodes;                /* n[0] n[1] (n[2]) */
    int32_t populations_per_node; /* 15 (2D) or 28 (3D) */
    int32_t bytes_per_population; /* 8, 4 or 2 (mixed layouts: 2 for the moving populations, 4 for the rest) */
    size_t  lattice_bytes;        /* bytes of one population lattice */
} vlbm_derived;

/* Fill *p with the parameters of Section 6.1: mu = 8, omega_rho = 6/5,
 * alpha_rho = 3/40, omega_q = 23/20 with alpha_q from nu (Prop. 1),
 * gamma = 1, rho_bar = 1, non-strict.  n has dim entries.  Never fails on a
 * non-null p. */
void vlbm_params_default(vlbm_params* p, int32_t dim, const int64_t* n, double dx, double nu, int32_t precision);

/* Validate *p and fill *out (may be NULL).  Host only: makes no CUDA call.
 * Returns VLBM_OK, VLBM_WSTABILITY, VLBM_EINVAL or VLBM_ESTABILITY.
 * Ranges: omega in (0, 2) (Section 2; 2 excluded by Prop. 1), alpha in
 * [0, 1/4] (2D) / [0, 1/6] (3D) (Lemma 1), gamma >= 1, dx, mu, rho_bar > 0. */
int vlbm_params_check(const vlbm_params* p, vlbm_derived* out);

/* Create a handle: validates *p, allocates two population lattices and the
 * scratch buffers on the current CUDA device, enqueued on `stream`
 * (a cudaStream_t, NULL for the legacy stream).  The lattice starts zeroed
 * (the rest state rho = rho_bar, q = 0); call vlbm_init to set a flow.
 * On failure *out is NULL and nothing is leaked. */
int vlbm_create(const vlbm_params* p, void* stream, vlbm_handle** out);

/* Release every buffer of h (after its stream's work completes).  NULL is a no-op. */
void vlbm_destroy(vlbm_handle* h);

/* Move all further work of h onto `stream`. */
int vlbm_set_stream(vlbm_handle* h, void* stream);

/* Initialise at equilibrium (end of Section 2) from a velocity field u
 * ([d][..][nx]) and an optional pressure-like potential phi ([..][nx],
 * NULL means 0): P(rho) = P(rho_bar) + dx^2 rho_bar phi (Prop. 1),
 * q = rho u, f = f^eq(rho, q).  Resets the step counter to 0. */
int vlbm_init(vlbm_handle* h, const void* u, const void* phi, int32_t dtype);

/* Advance nsteps >= 0 time steps (relaxation then transport each).  Enqueued
 * asynchronously unless VLBM_STEP_CHECK_FINITE is set (then it synchronises
 * and returns VLBM_EDIVERGED if any population is not finite). */
int vlbm_step(vlbm_handle* h, int64_t nsteps, int32_t flags);

/* Advance nsteps like vlbm_step and record, for every step s (0-based within
 * the call) with s % every == 0, the invariants of the state that step
 * produces (time step0 + s + 1: the moments of the transported populations,
 * which relaxation conserves) into history[(s / every) * 8 + i], in the
 * layout of vlbm_invariants.  The reduction is fused into the step kernel:
 * it reads no lattice data beyond what the step reads, and the kernel's
 * last block folds the partial sums into the record (one launch per
 * record).  history holds ceil(nsteps / every) records; it may be device
 * memory, pinned host memory (written asynchronously: valid once the
 * handle's stream has synchronised; page-locked memory mapped into the
 * device's address space is written by the step kernel itself, other
 * page-locked memory by a copy after each record) or pageable host memory
 * (the call synchronises before returning).  every >= 1; nsteps = 0
 * records nothing. */
int vlbm_step_record(vlbm_handle* h, int64_t nsteps, int64_t every, double* history);

/* Macroscopic fields at the current step: rho, u = q / rho and
 * phi = (P(rho) - P(rho_bar)) / (dx^2 rho_bar); any pointer may be NULL. */
int vlbm_macros(vlbm_handle* h, void* rho, void* u, void* phi, int32_t dtype);

/* Reduce the lattice in FP64 into out[8] (host or device pointer):
 *   { sum rho, sum q_x, sum q_y, sum q_z, E_kin = 1/2 sum |q|^2/rho dx^d,
 *     max |u|, number of nodes holding a non-finite population,
 *     sum (rho - rho_bar) }.
 * Sums run over finite nodes only, in a fixed order (deterministic). */
int vlbm_invariants(vlbm_handle* h, double* out);

/* Step counter and time t = step * dx^2 / mu.  Either pointer may be NULL. */
int vlbm_time(const vlbm_handle* h, int64_t* step, double* t);

/* Opaque checkpoint of h: a header (format, sizes, precision, step) followed
 * by the raw population lattice.  vlbm_state_bytes gives the size;
 * vlbm_set_state accepts only a checkpoint of an identical configuration
 * and restores the populations and the step counter bit for bit. */
size_t vlbm_state_bytes(const vlbm_handle* h);
int vlbm_get_state(vlbm_handle* h, void* dst, size_t bytes);
int vlbm_set_state(vlbm_handle* h, const void* src, size_t bytes);

/* Export the populations f*(t) as [k][l][..][nx] (k field, l velocity in the
 * order rest, +x, -x, +y, -y(, +z, -z)).  deviation = 0: absolute values;
 * deviation = 1: f - f^eq(rho_bar, 0), the quantity the FP32 and shifted
 * formats store (exact for those formats when dtype is wide enough). */
int vlbm_get_populations(vlbm_handle* h, void* dst, int32_t dtype, int32_t deviation);

/* Number of kernel launches this handle has issued (graph replays count
 * each kernel they contain). */
int vlbm_launch_count(const vlbm_handle* h, int64_t* count);

/* Tuning and test options.  VLBM_OPT_KERNEL selects the step kernel:
 * 0 = automatic (vectorised when n_x is a multiple of the nodes per lane:
 * 2D 4 (FP32, 16-bit formats) or 2 (FP64); 3D 2 or 1 (FP64)), 1 = one thread
 * per node (any size),
 * 2 = vectorised (VLBM_EINVAL when n_x does not allow it).  Both compute the
 * same arithmetic in the same order and agree to rounding (the compiler may fuse
 * a multiply and an add into one FMA in one kernel and not in the other). */
#define VLBM_OPT_KERNEL 0
/* VLBM_OPT_SPLIT_LANES: nodes per lane (2 or 4, default 4) of the vectorised 2D
 * kernel of the split formats; a tuning knob, same results up to FMA contraction. */
#define VLBM_OPT_SPLIT_LANES 1
/* VLBM_OPT_ROUNDING_16: rounding of the rest populations of the shifted 16-bit
 * formats (VLBM_FP16_SHIFTED, VLBM_BF16_SHIFTED; VLBM_EINVAL for the others):
 * 0 = to nearest (default), 1 = stochastic (unbiased; random bits from a hash of
 * node, field and step, so runs stay reproducible).  Under the parabolic scaling
 * a moment changes per step by much less than a 16-bit quantum: rounding to
 * nearest drops the change (a slowly evolving flow stops evolving), stochastic
 * rounding keeps it on average at the price of noise of about one quantum per
 * step.  FP32 storage always rounds its moment-carrying populations
 * stochastically (they are 2^13 times finer, so the noise is negligible). */
#define VLBM_OPT_ROUNDING_16 2
int vlbm_set_option(vlbm_handle* h, int32_t key, int64_t value);

/* Boundary conditions of a 2D lattice (Section 6.2.1, the Poiseuille test of
 * Section 6.2).  VLBM_BC_PERIODIC (the default): periodic wrap on every side.
 * VLBM_BC_CHANNEL: the ghost-cell conditions of the paper on the domain
 * [0, n_x dx] x [0, n_y dx]: ghost cells at distance dx/2 outside each side get
 * conserved moments from the two nearest interior cells of the current time
 * level -- left side: prescribed velocity (u_in(y), 0) (momentum
 * 2 rho_bar u_in - q of the adjacent cell) and linearly extrapolated density;
 * right side: prescribed pressure potential Phi_out (density
 * 2 rho_bar (1 + dx^2 Phi_out) - rho of the adjacent cell) and linearly
 * extrapolated momentum; lower and upper walls: zero velocity (momentum -q of
 * the adjacent cell) and extrapolated density -- and the population that
 * streams from a ghost cell into the domain is that cell's equilibrium (Eqs.
 * BCPoiseuilleLeftEquilibrium, BCPoiseuilleRightEquilibrium,
 * BCPoiseuilleLowerEquilibrium).  wall_correction = 1 adds at the walls the
 * non-equilibrium part of the same population at the adjacent interior cell
 * (Eq. BCPoiseuilleLowerEquilibriumPlusCorrection), which the paper shows is
 * needed for second order when omega_q != 1.
 * u_in: host array of n_y velocities u_x at the cell centres y = (j + 1/2) dx,
 * copied by the call (which synchronises the handle's stream).  Only 2D
 * lattices with VLBM_FP64 or VLBM_FP32 storage and at least 2 x 2 nodes
 * (VLBM_EINVAL otherwise).  A channel step is two kernel launches (ghost
 * populations, then the per-node stream-collide); vlbm_step_record is not
 * available with a channel (VLBM_EINVAL: step with vlbm_step and reduce with
 * vlbm_invariants).  Setting VLBM_BC_PERIODIC returns to the periodic step. */
#define VLBM_BC_PERIODIC 0
#define VLBM_BC_CHANNEL 1
typedef struct {
    int32_t kind;             /* VLBM_BC_PERIODIC or VLBM_BC_CHANNEL */
    int32_t wall_correction;  /* 1: non-equilibrium correction at the walls */
    double phi_out;           /* pressure potential Phi at the outlet x = n_x dx */
    const double* u_in;       /* host, n_y inflow velocities u_x(y) (VLBM_BC_CHANNEL) */
} vlbm_boundary;
int vlbm_set_boundary(vlbm_handle* h, const vlbm_boundary* bc);

/* Vorticity diagnostic of the current state: out[0] = sum over nodes of
 * |curl u|^2 dx^d, u = q / rho, with centred differences (periodic) of spacing
 * dx; in 2D the scalar vorticity d_x u_y - d_y u_x.  With the kinetic energy E of
 * vlbm_invariants it gives the energy balance of the incompressible limit,
 * -dE/dt = nu * sum |curl u|^2 dx^d (not an operation of the paper: a diagnostic
 * of its Navier-Stokes target).  The velocity is formed in FP32 in the handle's
 * staging buffer (allocated on first use), the differences and sums in FP64.
 * out: 1 double, host or device memory (host: the call synchronises the stream). */
int vlbm_vorticity_sq(vlbm_handle* h, double* out);

/* The reduction of vlbm_invariants for callers that cannot allocate device
 * memory: code running inside a pool or arena that owns all device memory,
 * in a real-time loop that may not take the allocator's locks or its implicit
 * synchronisation, or near the memory limit.  The paper has no counterpart;
 * it is an integration aid.  It needs no handle and allocates nothing: the
 * per-block partial sums live in a static device array of about 520 KiB that
 * each GPU loading the library keeps until the process exits.
 *   p       parameters of the lattice (checked like vlbm_params_check)
 *   lattice device pointer to one population lattice in a handle's storage
 *           layout: the vlbm_derived.lattice_bytes that follow the checkpoint
 *           header in a vlbm_get_state blob (the caller may keep that copy in
 *           its own device memory)
 *   out     8 doubles in the layout of vlbm_invariants; device memory, or host
 *           memory (then the call synchronises `stream` before returning)
 *   stream  cudaStream_t, NULL for the legacy stream
 * At most 8192 x 8192 = 67,108,864 nodes; larger lattices, a lattice that is
 * not device memory of the current device, a device `out` on another device
 * or bad parameters give VLBM_EINVAL; a CUDA error still pending from the
 * caller's earlier work gives VLBM_ECUDA (it is not cleared).  The first call on a device
 * looks up the static array's device address (cudaGetSymbolAddress): make
 * that first call before any stream capture.  All calls share the array, and
 * each writes every slot it later reads; calls whose kernels overlap on the
 * GPU (two streams or two host threads) race on it and must be serialised. */
int vlbm_invariants_noalloc(const vlbm_params* p, const void* lattice, double* out, void* stream);

/* ---- batched problems ----------------------------------------------------
 * Many independent periodic 2D problems advanced together: each has its own
 * vlbm_params (size, dx, viscosity, relaxation; dt = dx^2 / mu of its own),
 * all share one precision; any n[0] (a problem whose n[0] is not a multiple
 * of the format's vector width runs the per-node body, one node per lane).  A
 * vlbm_batch_step advances every problem by one of its own time steps with
 * one persistent kernel launch over a work list of (problem, row, segment)
 * items; runs of steps replay a captured CUDA graph, or run in one
 * cooperative launch (VLBM_STEP_PERSISTENT).  The arithmetic is that of a
 * single handle.  Not an operation of the paper: a way to run many of
 * its problems at once. */
typedef struct vlbm_batch vlbm_batch;

/* problems: `count` parameter sets (dim 2, same precision).  Allocates two
 * levels of all lattices (each 256-byte aligned) on the current device,
 * zeroed (rest state).  On failure *out is NULL. */
int vlbm_batch_create(const vlbm_params* problems, int32_t count, void* stream, vlbm_batch** out);
void vlbm_batch_destroy(vlbm_batch* b);

/* Initialise problem `problem` at equilibrium from u ([2][ny][nx]) and phi
 * ([ny][nx] or NULL), as vlbm_init; host or device pointers. */
int vlbm_batch_init(vlbm_batch* b, int32_t problem, const void* u, const void* phi, int32_t dtype);

/* Advance every problem by nsteps of its own time step (asynchronous).
 * flags & VLBM_STEP_PERSISTENT: one cooperative launch runs all nsteps (its
 * grid is the configured launch shape capped at the blocks that can be
 * resident together); its blocks wait for one another at every step
 * boundary, each wait bounded to about one second.  The call synchronises
 * and returns VLBM_ETIMEOUT if a wait gave up (the state is then partly
 * advanced).  The arithmetic, and so the state, is that of per-step
 * launches.  VLBM_STEP_TEST_TIMEOUT (with nsteps >= 2) makes the first
 * step boundary wait for one block more than the launch has, so every
 * block gives up after its bounded wait: the call returns VLBM_ETIMEOUT and
 * the handle stays usable.  Otherwise one launch per step (flags &
 * VLBM_STEP_NO_GRAPH) or replays of a captured graph of 32 launches. */
int vlbm_batch_step(vlbm_batch* b, int64_t nsteps, int32_t flags);

/* Macroscopic fields / invariants of one problem, as vlbm_macros / vlbm_invariants. */
int vlbm_batch_macros(vlbm_batch* b, int32_t problem, void* rho, void* u, void* phi, int32_t dtype);
int vlbm_batch_invariants(vlbm_batch* b, int32_t problem, double* out);

/* Launch shape of the step kernel: threads per block (128 or 256), blocks per
 * SM (1..16) and, for the split and shifted 16-bit formats, nodes per lane
 * (2 or 4; ignored for FP32 and FP64, which take 16-byte vectors). */
int vlbm_batch_set_config(vlbm_batch* b, int32_t threads, int32_t blocks_per_sm, int32_t lanes);

/* Time every candidate launch shape on `repeats` dry-run steps (they read the
 * current level and write the other without committing it, so the state is
 * unchanged), keep the fastest, and return it in config_out[3] =
 * {threads, blocks_per_sm, lanes} and its time per step in *best_ms (either
 * may be NULL).  Synchronises the batch's stream. */
int vlbm_batch_autotune(vlbm_batch* b, int32_t repeats, int32_t* config_out, double* best_ms);

/* Masked initialisation of equally sized 2D problems (same n, dx, gamma,
 * rho_bar) from one device state array states [count][channels][ny][nx] FP32:
 * every problem p with mask[p] != 0 (device uint8 array of count entries) is
 * set to the equilibrium of u = channels 0, 1 and phi = channel 2 (0 when
 * channels == 2), as vlbm_batch_init does for one problem.  One launch,
 * asynchronous.  VLBM_EINVAL for unequal problems or host pointers. */
int vlbm_batch_init_states(vlbm_batch* b, const float* states, int32_t channels, const uint8_t* mask);
/* Masked read-out into the same kind of array: u of problem p into channels
 * 0, 1 of states[p] and, when channels >= 3, phi into channel 2, for every p
 * with mask[p] != 0; other entries are left untouched.  One launch. */
int vlbm_batch_macros_states(vlbm_batch* b, float* states, int32_t channels, const uint8_t* mask);

/* Total nodes, steps taken and kernel launches issued; any pointer may be NULL. */
int vlbm_batch_info(const vlbm_batch* b, int64_t* nodes_total, int64_t* step, int64_t* launches);
const char* vlbm_batch_last_error(const vlbm_batch* b);

/* ---- tensor-core building block of the surrogate ---------------------------
 * D = A B^T on the fifth-generation tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation in tensor memory): A [M][K] and B [N][K] row-major BF16
 * device arrays (16-byte aligned), D [M][N] row-major FP32 device array.
 * M % 128 == 0, 16 <= N <= 256 with N % 16 == 0, K % 64 == 0.  *err_dev (device int) is set
 * to 1 if a bounded wait for the tensor core gave up.  Asynchronous on stream.
 * Not an operation of the paper: the GEMM the learned surrogate is built on. */
int vlbm_tc_gemm_bf16(const void* A, const void* B, float* D, int64_t M, int64_t N, int64_t K, int32_t* err_dev,
                      void* stream);

/* 3x3 convolution with periodic padding on the tensor cores (implicit GEMM):
 *   Y[b][y][x][co] = act(bias[co] + sum_{dy,dx,ci} W[co][3(dy+1)+(dx+1)][ci] X[b][y+dy][x+dx][ci])
 * with indices wrapped periodically.  X [B][H][W][cin] and Y, Z [B][H][W][cout]
 * are BF16 NHWC device arrays, W [cout][9][cin] BF16, bias [cout] FP32;
 * X, W, Y and Z 16-byte aligned (VLBM_EINVAL otherwise).
 * act = 1 applies GELU (tanh form, 0.5 x (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))))
 * and, when Z is not NULL, also stores the
 * pre-activation in Z; act = 0 stores the affine result.  (cin, cout) in
 * {16, 64} x {16, 64}.  *err_dev is set to 1 if a wait for the tensor core
 * gave up.  Asynchronous on stream. */
int vlbm_sur_conv3x3(const void* X, const void* W, const float* bias, void* Y, void* Z, int64_t B, int64_t H,
                     int64_t Wd, int32_t cin, int32_t cout, int32_t act, int32_t* err_dev, void* stream);

/* Weight and bias gradients of vlbm_sur_conv3x3, accumulated (+=) into
 *   G[co][3(dy+1)+(dx+1)][ci] += sum_{b,y,x} X[b][y+dy][x+dx][ci] dZ[b][y][x][co]
 *   Gb[co]                   += sum_{b,y,x} dZ[b][y][x][co]
 * (periodic indices) on the tensor cores.  X [B][H][W][cin], dZ [B][H][W][cout]
 * BF16 NHWC device arrays, 16-byte aligned; G [cout][9][cin] and Gb [cout] FP32 device arrays
 * that the caller zeroes first.  (cin, cout) in {(16,64), (64,64), (64,16)};
 * B H W < 2^31.  Asynchronous on stream; *err_dev as above. */
int vlbm_sur_conv3x3_wgrad(const void* X, const void* dZ, float* G, float* Gb, int64_t B, int64_t H, int64_t Wd,
                           int32_t cin, int32_t cout, int32_t* err_dev, void* stream);

/* ---- learned surrogate (an extension: the paper has no counterpart) ---------
 * A five-layer fully convolutional network with periodic 3x3 kernels, 64
 * hidden channels and GELU, mapping a coarse state u [B][C][H][W] (FP32,
 * device; C = channels, e.g. u_x, u_y and the pressure potential phi) to an
 * increment of the same shape.  The input is multiplied per channel by
 * in_scale before the network, its output by out_scale after it, so that
 * vlbm_sur_advance computes u + out_scale * net(in_scale * u).  Weights are
 * BF16 copies of FP32 master parameters, activations BF16, every product
 * accumulated in FP32 on the tensor cores.  Training minimises the mean
 * squared error of net(in_scale * u) against a target increment already
 * divided by out_scale, with Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8).
 * The handle owns all its device memory (parameters, Adam moments and
 * activations for max_batch states) and works on the stream given at creation. */
typedef struct vlbm_sur vlbm_sur;

/* Derived input channel: the periodic central-difference divergence of
 * channels 0, 1 (unit spacing), taken in FP32 before the input is rounded to
 * BF16.  It becomes input channel `channels`. */
#define VLBM_SUR_FEATURE_DIV 1
/* Divergence-free velocity increments: output channel 0 is a stream function
 * psi, the increment of channels 0, 1 is out_scale[0] (D_y psi, -D_x psi) with
 * periodic central differences D_y psi = (psi(y+1) - psi(y-1)) / 2 (rows y),
 * which the same differences see as exactly divergence-free; output channel 1
 * is unused.  Training targets of channels 0, 1 are the velocity increments
 * divided by out_scale[0]; the loss compares them with (D_y psi, -D_x psi), so
 * the network fits their solenoidal part. */
#define VLBM_SUR_FEATURE_CURL 2

/* 1 <= channels, channels + derived features <= 16, H W max_batch < 2^31.
 * features: an OR of VLBM_SUR_FEATURE_* (both need channels >= 2).  Seeded
 * initialisation (uniform, scaled by the fan-in), scales 1.  Synchronises. */
int vlbm_sur_create(int32_t H, int32_t W, int32_t channels, int32_t features, int32_t max_batch, uint64_t seed,
                    void* stream, vlbm_sur** out);
void vlbm_sur_destroy(vlbm_sur* s);
/* Per-channel input factors (host array of channels + derived features floats,
 * the derived ones last) and output factors (host array of `channels`
 * floats); NULL = all 1. */
int vlbm_sur_set_scaling(vlbm_sur* s, const float* in_scale, const float* out_scale);
/* Gaussian noise added to the network's inputs in vlbm_sur_train_step only
 * (after the input factors, so in units of the scaled inputs): standard
 * deviation sigma[c] per input channel (host array of channels + derived
 * features floats, >= 0; NULL = none), drawn from a counter-based generator
 * seeded by `seed`, a fresh draw for every step, pixel and channel.
 * Synchronises. */
int vlbm_sur_set_train_noise(vlbm_sur* s, const float* sigma, uint64_t seed);
/* Number of FP32 parameters: per layer the weights [cout][9][cin] then the
 * bias [cout], layers in order, with (cin, cout) = (16,64), (64,64), (64,64),
 * (64,64), (64,16); input channels beyond channels + derived features of the
 * first layer and output channels >= `channels` of the last are padding and
 * stay zero. */
int64_t vlbm_sur_num_params(const vlbm_sur* s);
/* du = net(in_scale * u) (no output scaling) for 1 <= batch <= max_batch
 * states; device pointers; asynchronous. */
int vlbm_sur_forward(vlbm_sur* s, const float* u, float* du, int32_t batch);
/* One surrogate step: u_next = u + out_scale * net(in_scale * u) (with
 * VLBM_SUR_FEATURE_CURL the velocity channels take the curl of channel 0, and
 * u_next must not alias u); otherwise u_next may alias u.  Asynchronous. */
int vlbm_sur_advance(vlbm_sur* s, const float* u, float* u_next, int32_t batch);
/* The scaled increment alone: du = u_next - u of vlbm_sur_advance (du must not
 * alias u).  Asynchronous. */
int vlbm_sur_increment(vlbm_sur* s, const float* u, float* du, int32_t batch);
/* One Adam step on the mean squared error of net(in_scale * u) against target
 * (both [batch][C][H][W] FP32 device arrays) with learning rate lr.  When
 * loss is not NULL the loss before the update is written there (host float)
 * and the call synchronises; otherwise it is asynchronous. */
int vlbm_sur_train_step(vlbm_sur* s, const float* u, const float* target, int32_t batch, float lr, float* loss);
/* Copy the FP32 parameters (or the gradients of the last train step) to dst;
 * set_params also resets Adam's moments.  Any pointer kind; synchronise. */
int vlbm_sur_get_params(vlbm_sur* s, float* dst);
int vlbm_sur_get_grads(vlbm_sur* s, float* dst);
int vlbm_sur_set_params(vlbm_sur* s, const float* src);
/* VLBM_ETIMEOUT if a wait for the tensor core gave up since creation; synchronises. */
int vlbm_sur_status(vlbm_sur* s);

/* ---- field utilities of the surrogate's data path (not operations of the paper)
 * Average pooling of in [B][C][H factor][W factor] to out [B][C][H][W], FP32
 * device arrays (the coarse-graining of fine lattice fields). */
int vlbm_field_pool(const float* in, float* out, int64_t B, int64_t C, int64_t H, int64_t W, int32_t factor,
                    void* stream);
/* Training pairs from a store of consecutive states snaps [n][C][H][W]:
 * u[b] = snaps[idx[b]], target[b][c] = (snaps[idx[b]+1][c] - snaps[idx[b]][c]) * inv_scale[c],
 * idx a device int64 array of batch entries with idx[b] + 1 < n (not
 * checked), inv_scale a host array of C floats. */
int vlbm_sur_gather_pairs(const float* snaps, const int64_t* idx, float* u, float* target, int32_t channels,
                          int64_t H, int64_t W, int32_t batch, const float* inv_scale, void* stream);
/* Per-state statistics of the velocity channels 0, 1 of u [batch][channels][H][W]
 * (periodic, unit spacing, central differences) into out [batch][3] FP64
 * device array: kinetic energy sum |u|^2 / 2, sum of squared divergence, sum
 * of |grad u|^2.  The surrogate's rollout check reads these.  Asynchronous. */
int vlbm_field_stats(const float* u, double* out, int32_t batch, int32_t channels, int64_t H, int64_t W,
                     void* stream);
/* The surrogate rollout's per-state check on the device (not an operation of
 * the paper; the fallback rule of the learned surrogate).  stats and prev
 * [n][3] FP64 device arrays as vlbm_field_stats writes them, for the new
 * states and the states they were advanced from; e0 [n] the starting
 * energies, r_max [n] the largest admitted divergence-to-gradient ratios.
 * State b fails when |E/E_prev - 1| > step_tol, |E/E_0 - 1| > drift_tol or
 * sqrt(D / max(G, 1e-300)) > r_max[b], NaN counting as a failure; then
 * mask[b] = 1 (else 0) and counts[b] += 1.  counts [n + 3] int64 device array:
 * per-state failures, then the failing tests (energy step, energy drift,
 * divergence), accumulated.  Asynchronous on stream; no host round trip. */
int vlbm_sur_rollout_check(const double* stats, const double* prev, const double* e0, const double* r_max, int32_t n,
                           double step_tol, double drift_tol, uint8_t* mask, int64_t* counts, void* stream);
/* Per-field error sums over the first n FP32 values of nfields fields that
 * lie ld values apart (device arrays a, b): out[f][0] = sum (a - b)^2,
 * out[f][1] = sum b^2, FP64 device array out [nfields][2].  Asynchronous. */
int vlbm_field_diff_norms(const float* a, const float* b, double* out, int32_t nfields, int64_t n, int64_t ld,
                          void* stream);

/* Kernels launched by the surrogate and field-utility entry points above since
 * the library was loaded (all handles, all threads). */
int64_t vlbm_sur_launch_count(void);

/* Static text of a status code; message of the last failure of h. */
const char* vlbm_strerror(int code);
const char* vlbm_last_error(const vlbm_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* VLBM_H */
