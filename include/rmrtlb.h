/*
 * rmrtlb.h -- C ABI of the GB300 rectangular MRT lattice Boltzmann step.
 *
 * The library advances populations of the rectangular multiple-relaxation-
 * time lattice Boltzmann method (RMRT-LB) of Chai, Yuan & Shi (arXiv
 * 2206.00366) on rD2Q9, rD3Q19 and rD3Q27 lattices with unequal spacings
 * dx, dy, dz.  One time step is the forced moment-space collision of
 * Eq. (2-2-3),
 *
 *     fbar(x + c_j dt, t + dt) = M^-1 [ mbar - S (mbar - m^eq)
 *                                       + dt (m_G + (I - S/2) m_F) ],
 *
 * with m = M f the raw moments of Eq. (5-2), the rectangular equilibrium
 * g^eq(A, B, M) of Eqs. (3-3)/(3-4), the block relaxation matrix S of
 * Eq. (5-1) whose second-order block comes from the shear and bulk
 * viscosities (Eqs. 4-27, 4-31, 5-8-1), and periodic propagation (Eq. 2-2b).
 * The central-moment variant relaxes N(u) m with the same block rates
 * (Eqs. 5-1-1, 5-1-2).
 *
 * Conventions shared by every entry point:
 *   - Every function returns RMRTLB_OK (0) or a negative status; no C++
 *     exception crosses the ABI.  rmrtlb_strerror() names a status.
 *   - Fields are FP64, structure-of-arrays, x fastest: a scalar field has
 *     nx*ny*nz values at index (z*ny + y)*nx + x; a vector field stores its
 *     d components as d consecutive scalar planes; populations store q
 *     planes in the velocity order given by rmrtlb_lattice_info().  2-D
 *     lattices take nz = 1.
 *   - Field and population pointers may be host or device memory; the
 *     library finds out which (cudaPointerGetAttributes).  Host data is
 *     staged through the workspace with cudaMemcpyAsync on the handle's
 *     stream, and the call returns after the host buffer is no longer
 *     needed (it synchronises the stream for host pointers only).
 *   - Device work is issued on the CUDA stream given at creation; calls
 *     with device pointers return without synchronising.
 *   - The library allocates no device memory: the caller passes one
 *     device workspace of rmrtlb_workspace_bytes() bytes, which it owns,
 *     keeps alive until rmrtlb_destroy(), and frees afterwards.
 *   - Lattice units: c_alpha = dx_alpha / dt is the lattice speed along
 *     axis alpha; discrete velocities are c_j = e_j * c with
 *     e_j in {-1, 0, 1}^d.
 */
#ifndef RMRTLB_H
#define RMRTLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define RMRTLB_OK         0
#define RMRTLB_EINVAL    (-1)  /* bad argument: lattice, size, negative weight,
                                  c_s^2 >= min c_a^2, rate outside (0, 2) */
#define RMRTLB_ENOMEM    (-2)  /* workspace smaller than rmrtlb_workspace_bytes */
#define RMRTLB_ECUDA     (-3)  /* a CUDA runtime call failed */
#define RMRTLB_EUNSTABLE (-4)  /* NaN/Inf, density <= 0 or |u| >= c_s seen by
                                  the last check step */
#define RMRTLB_ETOOBIG   (-5)  /* input larger than a fixed-size internal
                                  buffer allows */
#define RMRTLB_ETIMEOUT  (-6)  /* a bounded device-side wait gave up: the
                                  kernel skipped its outputs and returned */

/* --------------------------------------------------------------- choices */
/* Lattices of Sec. III.  rD2Q5 and rD3Q7 (Remark I: rest and axis
 * directions, omega_a = c_s^2 / (2 c_a^2), default c_s^2 = min c_a^2 / 3 and
 * min c_a^2 / 4 respectively) carry only the simplified NCDE kinds; their
 * moment basis is 1, the first powers and the squares of each axis. */
enum rmrtlb_lattice {
    RMRTLB_D2Q9 = 0, RMRTLB_D3Q19 = 1, RMRTLB_D3Q27 = 2,
    RMRTLB_D2Q5 = 3, RMRTLB_D3Q7 = 4
};

/* Equilibrium kind (which conservation law the step solves).
 *  NSE          f^eq = g^eq(rho, rho u, rho u u)              Eq. (NSEfeq)
 *  NSE_HELUO    f^eq = g^eq(rho, rho0 u, rho0 u u)            Sec. IV Remark IV
 *  NCDE_LINEAR  f^eq = g^eq(phi, u phi, u u phi)              Eq. (4-14) with
 *                                                             D = phi I, beta = 1,
 *                                                             C = int B'B' dphi
 *  NCDE_QUAD    f^eq = g^eq(phi, u phi^2/2, u u phi^3/3)      same, B = u phi^2/2
 *  NCDE_SIMPLE_LINEAR  f^eq = g^eq(phi, u phi, 0)             Eq. (4-16): C = 0,
 *  NCDE_SIMPLE_QUAD    f^eq = g^eq(phi, u phi^2/2, 0)         G = g^eq(0, (I - S_1/2)
 *                                                             dB/dt, 0), F = omega S
 * For the NCDE kinds u is the constant advection velocity params.adv.  The
 * simplified kinds take dB/dt = (B(t) - B(t - dt)) / dt from a per-node
 * history of B kept in the workspace; the first step after create,
 * rmrtlb_init_equilibrium or rmrtlb_set_populations uses dB/dt = 0. */
enum rmrtlb_eq_kind {
    RMRTLB_EQ_NSE = 0,
    RMRTLB_EQ_NSE_HELUO = 1,
    RMRTLB_EQ_NCDE_LINEAR = 2,
    RMRTLB_EQ_NCDE_QUAD = 3,
    RMRTLB_EQ_NCDE_SIMPLE_LINEAR = 4,
    RMRTLB_EQ_NCDE_SIMPLE_QUAD = 5
};

/* Moment basis of the relaxation, Mbar = N M (Eqs. 5-1-1, 5-1-2): raw
 * moments (Eq. 5-2, N = I); central moments about the local velocity
 * (N = N(u)); Hermite moments, the tensor products of P_0 = 1, P_1 = c,
 * P_2 = c^2 - c_s^2 per axis; central-Hermite moments, the same polynomials
 * of c - u.  The relaxation matrix Sbar has the same blocks in every basis
 * (rates of Eq. 4-31, S_2 block of Eq. 5-8-1, s_free for orders >= 3). */
enum rmrtlb_basis {
    RMRTLB_BASIS_RAW = 0,
    RMRTLB_BASIS_CENTRAL = 1,
    RMRTLB_BASIS_HERMITE = 2,
    RMRTLB_BASIS_CENTRAL_HERMITE = 3
};

/* Population storage.  Every kind stores the deviation fbar_j - omega_j rho0;
 * F64 computes in FP64, the others in FP32.
 *   F16:   IEEE binary16 of the deviation times the power of two nearest
 *          1/omega_j (exact to apply and undo, keeps small-weight
 *          populations out of FP16's subnormals).
 *   BF16:  bfloat16 of the deviation, unscaled (FP32's exponent range).
 *   E3M12: a 16-bit float with a sign, 3 exponent bits and 12 mantissa
 *          bits, with subnormals, of the deviation times the same power of
 *          two as F16, in a range R set by rmrtlb_params.storage_range (a
 *          power of two, default 2 for the NSE and 8 for the NCDE): 4x
 *          FP16's resolution for scaled magnitudes in [R/128, R), a fixed
 *          spacing of R * 2^-19 below.  Magnitudes that round beyond R
 *          saturate; the check then reports RMRTLB_EUNSTABLE with flag 8.
 * The 16-bit kinds round stochastically in rmrtlb_step (the rounding
 * error has mean zero and is not repeated from step to step; the random
 * bits come from a counter-based generator of the step index and the node,
 * so runs are reproducible) and to nearest even when populations are set
 * or initialised. */
enum rmrtlb_storage {
    RMRTLB_ST_F64 = 0,
    RMRTLB_ST_F32 = 1,
    RMRTLB_ST_F16 = 2,
    RMRTLB_ST_BF16 = 3,
    RMRTLB_ST_E3M12 = 4
};

/* ------------------------------------------------------------ parameters */
typedef struct {
    double cs2;          /* c_s^2 (Sec. III, c_{s alpha} = c_s); <= 0 selects
                            min_alpha c_alpha^2 / 3 */
    double rho0;         /* reference density (NSE) or phi (NCDE) of the stored
                            deviation; also rho0 of the He-Luo equilibrium */
    double nu;           /* NSE kinematic viscosity: gives s_{alpha beta} and
                            s_{s alpha} through Eq. (4-31a) */
    double nu_bulk;      /* NSE bulk viscosity: gives s_{b alpha}, Eq. (4-31b) */
    double s_free;       /* rate of every moment not fixed by the model (order
                            >= 3 for the NSE, order >= 2 for the NCDE) */
    double s0, s1;       /* NSE rates of orders 0 and 1 (they do not enter the
                            unforced NSE); <= 0 selects s_free */
    double s_shear[3];   /* > 0 overrides s_{s alpha} from nu */
    double s_bulk[3];    /* > 0 overrides s_{b alpha} from nu_bulk */
    double s_off[3];     /* > 0 overrides s_xy, s_xz, s_yz from nu */
    double diffusivity;  /* NCDE: K = diffusivity * I through S_1 = I / tau,
                            tau = diffusivity / (c_s^2 dt) + 1/2 (Eq. 4-10) */
    double adv[3];       /* NCDE constant advection velocity */
    double force[3];     /* NSE body force Fbar (uniform), Eq. (NSE) */
    double source;       /* NSE mass source Sbar or NCDE source S (uniform) */
    int check_every;     /* rmrtlb_step runs the FP64 check (mass, momentum,
                            residual, stability flags) every check_every
                            steps; 0 disables it */
    double storage_range;/* E3M12 storage: the scaled deviation
                            (fbar_j - omega_j rho0) * 2^round(-log2 omega_j)
                            is stored in a range that ends at the power of two
                            at or above storage_range (values that round
                            beyond it saturate and the check reports flag 8);
                            the format's resolution scales with the range.
                            <= 0 selects 2 for the NSE kinds (flows up to a
                            Mach number of about 0.3) and 8 for the NCDE
                            kinds (phi - rho0 of order 1).  Ignored by the
                            other storages. */
    long long node_offset;/* index of this grid's first node within a larger
                            grid it is a slab of (rmrtlb_halo_pack): the
                            16-bit stochastic rounding draws its random bits
                            from the step and the node's index in the larger
                            grid, so slabs reproduce the whole grid's run
                            bit for bit.  0 for a grid of its own. */
} rmrtlb_params;

typedef struct rmrtlb_solver* rmrtlb_t;   /* opaque, library-owned */

/* Name of a status code (static string, never NULL). */
const char* rmrtlb_strerror(int status);

/* Velocity set of a lattice.  Writes q and d; when e is not NULL it
 * receives q*3 integers e_j = (e_x, e_y, e_z) in {-1,0,1}, in the order
 * used for population planes: rD2Q9 as Eq. (3-1), rD3Q27 as Eq. (3-2) (the
 * xz block read as (1,0,1), (-1,0,1), (-1,0,-1), (1,0,-1)), rD3Q19 as the
 * first 19 of rD3Q27 (Sec. III).  Host only; touches no GPU. */
int rmrtlb_lattice_info(int lattice, int* q, int* d, int* e);

/* Bytes of device workspace rmrtlb_create needs for this grid and storage:
 * two population lattices, a staging area for host transfers, the residual
 * snapshot and the reduction scratch.  Host only. */
int rmrtlb_workspace_bytes(int lattice, int nx, int ny, int nz, int storage,
                           size_t* bytes);

/* Derive every constant of the step on the host and bind a solver to the
 * caller's workspace.  Constants: c_alpha = d_alpha / dt, c_s^2, weights
 * (Eq. 3-3-5 for rD2Q9; Eq. 3-3-8 for rD3Q27 with omega_19 =
 * c_s^6 / (8 c1^2 c2^2 c3^2); omega_19 = 0 for rD3Q19), rates from nu and
 * nu_bulk (Eq. 4-31), the dense S_2 block by Sherman-Morrison (Eq. 5-8-1).
 * Fails with RMRTLB_EINVAL for a negative weight, c_s^2 >= min c_alpha^2 or
 * a rate outside (0, 2); RMRTLB_ENOMEM if workspace_bytes is too small.
 * workspace: device pointer, 256-byte aligned, owned by the caller.
 * stream: a cudaStream_t (NULL = legacy default stream).  The populations
 * are left undefined: call rmrtlb_init_equilibrium or
 * rmrtlb_set_populations next.  Launches nothing. */
int rmrtlb_create(rmrtlb_t* solver, int lattice, int nx, int ny, int nz,
                  double dx, double dy, double dz, double dt,
                  const rmrtlb_params* params, int eq_kind, int basis,
                  int storage, void* workspace, size_t workspace_bytes,
                  void* stream);

/* Release the handle (not the workspace).  NULL is accepted. */
int rmrtlb_destroy(rmrtlb_t solver);

/* Host copy of the derived constants, for inspection:
 * out[0] = c_s^2, out[1..3] = c_alpha, out[4..30] = omega_j (q used),
 * out[31] = s0, out[32..34] = S_1 diagonal, out[35..43] = S_2 diagonal
 * block (row major, d x d used), out[44..46] = s_xy, s_xz, s_yz,
 * out[47] = s_free.  n is the capacity of out (>= 48). */
int rmrtlb_get_constants(rmrtlb_t solver, double* out, int n);

/* fbar = f^eq(rho, u) at every node (Eq. NSEfeq / Eq. 4-14; no
 * non-equilibrium part).  rho: scalar field (phi for the NCDE);
 * u: d planes (ignored for the NCDE).  Resets the step counter. */
int rmrtlb_init_equilibrium(rmrtlb_t solver, const double* rho, const double* u);

/* Set / read the populations fbar_j(x, t) of the current time (after
 * propagation, before collision), q planes in rmrtlb_lattice_info order.
 * set rounds to the storage type. */
int rmrtlb_set_populations(rmrtlb_t solver, const double* f);
int rmrtlb_get_populations(rmrtlb_t solver, double* f);

/* Advance n time steps (n >= 0), each one fused kernel: pull-propagation
 * gather (Eq. 2-2b), moments, macroscopic fields (Eq. 2-4-1/2-4-2),
 * equilibrium and forcing moments, relaxation (Eq. 2-2-3), inverse
 * transform, store.  Asynchronous on the solver's stream.  When
 * params.check_every > 0 the FP64 check runs after every multiple of it. */
int rmrtlb_step(rmrtlb_t solver, int n);

/* Macroscopic fields of the current populations (Eq. 2-4-1 / 2-4-2):
 * rho (or phi) one plane, u d planes (the advection velocity for the
 * NCDE).  Either pointer may be NULL. */
int rmrtlb_moments(rmrtlb_t solver, double* rho, double* u);

/* Local viscous stress and strain rate of the current state, NSE kinds
 * only (RMRTLB_EINVAL otherwise), Eqs. (4-32) and (4-33): with
 *   X = sum_k c_k c_k f_k^ne + (dt/2)(u Fbar + Fbar u + c_s^2 Sbar I),
 *   stress_ab = K_mu,ab (d_a u_b + d_b u_a) = -(1 - s_ab/2) X_ab,
 *   strain_ab = (d_a u_b + d_b u_a)/2 = stress_ab / (2 K_mu,ab),
 * every product entry by entry, s_aa = s_sa, s_ab the off-diagonal rates,
 * K_mu of Eq. (4-29a) at the local density, f^ne from the node's own
 * populations (no finite differences).  Each output is d(d+1)/2 FP64
 * planes of nz*ny*nx in the order xx, yy, (zz), xy, (xz, yz), DEVICE
 * memory (RMRTLB_EINVAL for a host pointer); either may be NULL.
 * Asynchronous on the solver's stream. */
int rmrtlb_stress(rmrtlb_t solver, double* stress, double* strain_rate);

/* Run the FP64 check on the current populations now and return, after
 * synchronising the stream:
 *   out[0] total mass sum rho (or sum phi)     out[1..3] total momentum
 *   out[4] kinetic energy sum rho |u|^2 / 2    out[5] residual
 *          ||u - u_prev||_2 / ||u||_2 against the previous check (-1 if
 *          there was none)                     out[6] step counter
 *   out[7] flags: 1 NaN/Inf, 2 density <= 0, 4 |u| >= c_s, 8 an E3M12
 *          population saturated (scaled magnitude 8 or more).
 * Returns RMRTLB_EUNSTABLE when a flag is set (out is still filled). */
int rmrtlb_stats(rmrtlb_t solver, double out[8]);

/* Result of the last check that rmrtlb_step ran (same layout as
 * rmrtlb_stats; out[6] = -1 if none ran yet).  Synchronises the stream. */
int rmrtlb_last_check(rmrtlb_t solver, double out[8]);

/* ------------------------------------------------------ batched cavities */
/* Many independent lid-driven cavities advanced together on one lattice
 * (rD2Q9, rD3Q19 or rD3Q27; raw or central moments): each a closed box of
 * nx x ny (x nz) nodes with half-way bounce-back walls half a spacing
 * outside the first and last node of every axis; the lid is the wall beyond
 * the last node of the last axis (y = ny - 1 on rD2Q9, z = nz - 1 on the
 * 3-D lattices) and moves along +x with lid_u.  A population whose source
 * x - e_j lies outside the box is the node's own post-collision population
 * in the opposite direction; one whose source lies beyond the lid gains
 * 2 omega_j rho0 (c_j . U) / c_s^2, the linear term of the REDF (Eq. 3-3).
 * Every node collides as in rmrtlb_step (Eq. 2-2-3, unforced NSE, the
 * central variant of Eq. 5-1-2 with basis RMRTLB_BASIS_CENTRAL), with its
 * domain's own spacing, c_s^2 (<= 0: the smallest spacing squared / 3),
 * weights (Sec. III) and rates (Eq. 4-31, Eq. 5-8-1).  The paper has no
 * boundaries; the wall rule is the standard half-way bounce-back. */
typedef struct {
    int nx, ny, nz;      /* nz = 1 on rD2Q9 */
    double dx, dy, dz;   /* spacings; lattice units, dt = 1 (dz unused on rD2Q9) */
    double nu, nu_bulk;  /* kinematic and bulk viscosity */
    double s_free;       /* rate of every moment of order >= 3 */
    double lid_u;        /* lid velocity (along +x) */
    double cs2;          /* <= 0 selects the smallest spacing squared / 3 */
} rmrtlb_domain;

typedef struct rmrtlb_batch* rmrtlb_batch_t;

/* Workspace bytes for these domains on `lattice` (RMRTLB_D2Q9, _D3Q19,
 * _D3Q27), storage RMRTLB_ST_F32 or _F64.  RMRTLB_EINVAL for a bad lattice,
 * storage or size (nz != 1 on rD2Q9, more than 65535 domains or 2^31 row
 * tiles).  Host only. */
int rmrtlb_batch_workspace_bytes(int lattice, int ndomains, const rmrtlb_domain* domains,
                                 int storage, size_t* bytes);

/* Bind a batch to the caller's workspace (device, 256-byte aligned, owned
 * by the caller).  basis: RMRTLB_BASIS_RAW or _CENTRAL.  Every domain starts
 * at rest (rho0, u = 0).  Every check_every steps (rounded up to even) the
 * FP64 residual ||u(t) - u(t - check_every)||_2 / ||u(t)||_2 of each domain
 * is formed; a domain whose residual falls below tol retires: it is no
 * longer stepped and keeps its state.  With a non-NULL stream, each chunk
 * of check_every steps plus its check is captured once as a CUDA graph and
 * replayed; the legacy NULL stream launches directly (capture needs a
 * created stream).  The tile list starts with 128-node single-row tiles
 * (see rmrtlb_batch_tune).  RMRTLB_EINVAL for invalid rates or weights of a
 * domain (as rmrtlb_create), RMRTLB_ENOMEM for a short workspace. */
int rmrtlb_batch_create(rmrtlb_batch_t* batch, int lattice, int basis, int ndomains,
                        const rmrtlb_domain* domains, int storage, double rho0,
                        int check_every, double tol, void* workspace,
                        size_t workspace_bytes, void* stream);
int rmrtlb_batch_destroy(rmrtlb_batch_t batch);

/* Every domain back at rest, active, step 0. */
int rmrtlb_batch_reset(rmrtlb_batch_t batch);

/* Autotuner: time `steps` steps with each launch shape — tile width 32,
 * 64, 128 or 256 nodes times 1, 2 or 4 rows per block, and for FP32
 * storage nodes per thread 1 or 0 (automatic) — keep the fastest, then
 * reset.  Nodes per thread: 1, a thread per node; 2 (FP32 only), two nodes
 * per thread collided together in packed FP32 arithmetic; 0 (automatic,
 * FP32 only), two while the domains being stepped hold at least twice as
 * many nodes as the GPU has resident threads, else one (a thread per node
 * finishes a step sooner when the batch, or what is left of it, is too
 * small to fill the GPU).  Writes the chosen width, rows and nodes per
 * thread (any pointer may be NULL).  The batch starts with 128 x 1 tiles
 * and the automatic mode (FP32) or one node per thread (FP64). */
int rmrtlb_batch_tune(rmrtlb_batch_t batch, int steps, int* tile_width, int* tile_rows,
                      int* nodes_per_thread);

/* Set the launch shape directly (the tuner's choices, e.g. from an earlier
 * run): tile_width 32, 64, 128 or 256; tile_rows 1, 2 or 4;
 * nodes_per_thread 1, or 2 or 0 with FP32 storage (see rmrtlb_batch_tune).
 * The state is kept.  RMRTLB_EINVAL for any other value. */
int rmrtlb_batch_set_launch(rmrtlb_batch_t batch, int tile_width, int tile_rows, int nodes_per_thread);

/* Advance every active domain n steps (asynchronous). */
int rmrtlb_batch_step(rmrtlb_batch_t batch, int n);

/* Advance until no domain is stepping (all converged or unstable) or
 * max_steps steps were issued; the state flags are read every 8 checks, so
 * up to 8 * check_every steps are issued after the last domain retired
 * (retired domains are skipped by the kernels).  *steps_done = steps
 * issued by this call.  Synchronises. */
int rmrtlb_batch_run(rmrtlb_batch_t batch, long long max_steps, long long* steps_done);

/* Per-domain arrays (any may be NULL): residual of the last check (-1
 * before the second check), step at which the domain retired (-1 while
 * stepping), state: 1 stepping, 0 converged (residual < tol), -1 unstable
 * (a non-finite velocity or |u| >= c_s at a check: retired so that it
 * cannot spoil the batch); *steps_done = steps issued.  Synchronises. */
int rmrtlb_batch_status(rmrtlb_batch_t batch, double* residual,
                        long long* steps_to_converge, int* active,
                        long long* steps_done);

/* Populations fbar_j(x, t) of one domain, q FP64 planes of nz*ny*nx (x
 * fastest) in rmrtlb_lattice_info order, host or device memory.
 * Synchronise. */
int rmrtlb_batch_set_populations(rmrtlb_batch_t batch, int domain, const double* f);
int rmrtlb_batch_get_populations(rmrtlb_batch_t batch, int domain, double* f);

/* Start one domain from macroscopic fields: rho one plane, u d planes
 * (FP64, host or device).  fbar = f^eq(rho, u) (Eq. NSEfeq); with
 * with_noneq != 0 the non-equilibrium part of Eq. (fne) is added, with
 * m_2^ne from Eq. (4-35): m_2^ne_aa = -rho (c_a^2 - c_s^2) dt (du_a/dx_a)
 * / s_sa and m_2^ne_ab = -rho c_s^2 dt (du_a/dx_b + du_b/dx_a) / s_ab,
 * the velocity gradients by central differences (one-sided at the first and
 * last node of an axis).  The domain's state flag is unchanged.
 * Synchronises. */
int rmrtlb_batch_init_fields(rmrtlb_batch_t batch, int domain, const double* rho,
                             const double* u, int with_noneq);

/* rho (one plane) and u (d planes) of one domain; host or device; either
 * may be NULL.  Synchronises. */
int rmrtlb_batch_fields(rmrtlb_batch_t batch, int domain, double* rho, double* u);

/* ------------------------------------------------ slab decomposition */
/* A periodic grid cut into slabs along its slowest axis (y on rD2Q9 and
 * rD2Q5, z on the 3-D lattices), one solver per slab, created with the
 * slab's own extent and periodic like any grid.  Propagation (Eq. 2-2b)
 * moves the populations with e_axis = +1 out of a slab's last plane into
 * the next slab's first, and those with e_axis = -1 the other way.  With
 * pull streaming a solver keeps each post-collision population at its own
 * node, and its first plane reads the e = +1 ones through the periodic
 * wrap from its own last plane, which no other node of the slab reads
 * (likewise e = -1 at the other end).  So after every rmrtlb_step(solver, 1)
 * a slab hands those planes round the ring of slabs:
 *   rmrtlb_halo_pack(s, up, down)   up   <- last plane, e_axis = +1 populations
 *                                   down <- first plane, e_axis = -1 populations
 *   send up to the next slab and down to the previous one (periodic ring)
 *   rmrtlb_halo_unpack(s, from_below, from_above)
 *                                   the previous slab's up buffer -> the last
 *                                   plane's e = +1 slots; the next slab's down
 *                                   buffer -> the first plane's e = -1 slots
 * after which the slabs together hold exactly the single grid's state.  A
 * single slab (no neighbours) needs no exchange.  Initialisation needs
 * none either (rmrtlb_init_equilibrium and rmrtlb_set_populations place
 * every value where its own node reads it).  Buffers: device memory of
 * rmrtlb_halo_bytes each (crossing directions in increasing j, one plane
 * each, x fastest, storage type), caller-owned; pack and unpack are
 * asynchronous on the solver's stream.  RMRTLB_EINVAL for NULL or host
 * buffers. */
int rmrtlb_halo_bytes(rmrtlb_t solver, size_t* bytes);
int rmrtlb_halo_pack(rmrtlb_t solver, void* up, void* down);
int rmrtlb_halo_unpack(rmrtlb_t solver, const void* from_below, const void* from_above);

/* One step in two parts, for overlapping a slab's halo exchange with its
 * interior (the populations that cross a face only enter the two planes
 * next to it).  Along the slab axis (y on rD2Q9 / rD2Q5, z on the 3-D
 * lattices) of n planes, rmrtlb_step_interior steps planes 2 .. n - 3: it
 * reads only planes 1 .. n - 2 of the current populations and writes only
 * the other lattice, so it may run while rmrtlb_halo_pack's buffers are in
 * flight and before rmrtlb_halo_unpack.  rmrtlb_step_boundary then steps
 * every plane the step has not stepped yet (planes 0, 1, n - 2, n - 1, or
 * all of them without an interior part) and completes the step exactly as
 * rmrtlb_step does (counter, periodic check); rmrtlb_step after an interior
 * part does the same.  The two parts give bitwise the step of rmrtlb_step.
 * With n < 5 the interior part steps nothing.  rmrtlb_step_interior twice
 * without completing the step, RMRTLB_EINVAL.  Asynchronous on the
 * solver's stream. */
int rmrtlb_step_interior(rmrtlb_t solver);
int rmrtlb_step_boundary(rmrtlb_t solver);

/* Run the periodic FP64 check now, on the current state, into the record
 * that rmrtlb_last_check and rmrtlb_check_sums read (the residual is taken
 * against the previous check's snapshot, which this call replaces), as
 * rmrtlb_step does every check_every steps.  For slabs, which must check
 * after their exchange: create them with check_every = 0 and call this
 * after rmrtlb_halo_unpack.  Asynchronous on the solver's stream. */
int rmrtlb_check(rmrtlb_t solver);

/* Raw sums of the last periodic check, for a reduction over slabs:
 *   out[0] sum rho (or phi)   out[1..3] momentum   out[4] kinetic energy
 *   out[5] sum |u - u_prev|^2 (-1 if the check had no previous snapshot)
 *   out[6] sum |u|^2          out[7] flags
 * The residual of the whole grid is sqrt(sum out[5] / sum out[6]) over the
 * slabs.  No check yet: zeros with out[6] = -1.  Synchronises the stream. */
int rmrtlb_check_sums(rmrtlb_t solver, double out[8]);

/* ------------------------------------------------ checkpoint / resume */
/* The paper has no counterpart.  A solver's state as one self-describing
 * blob: a header (format version, grid, storage, basis, equilibrium kind,
 * the step counter, the periodic check's bookkeeping, and every constant
 * the step derives from the parameters, as a fingerprint), then the
 * population codes exactly as stored, the residual snapshot of the last
 * check (if any), the simplified NCDE's B(t - dt) planes (that kind only)
 * and the last check's sums and flag word.  Loading it into a solver
 * created with the same lattice, grid, storage, basis, kind and parameters
 * and stepping on gives bitwise the same populations and checks as the
 * uninterrupted run (the 16-bit stochastic rounding draws its bits from
 * the step counter and the node index, both restored).
 *
 * rmrtlb_state_bytes: the blob's size for the solver's current state (it
 * grows by the snapshot once a check has run).  Host only.
 * rmrtlb_save_state: writes the blob to dst (host or device memory of at
 * least rmrtlb_state_bytes bytes, caller-owned); synchronises the stream.
 * rmrtlb_load_state: restores the state from src (host or device memory);
 * RMRTLB_EINVAL, with the solver unchanged, if the blob is not a state
 * blob, is shorter than its sections, or was saved from a solver with
 * another lattice, grid, storage, basis, kind, node_offset or any other
 * constant;
 * synchronises the stream. */
int rmrtlb_state_bytes(rmrtlb_t solver, size_t* bytes);
int rmrtlb_save_state(rmrtlb_t solver, void* dst, size_t bytes);
int rmrtlb_load_state(rmrtlb_t solver, const void* src, size_t bytes);

/* ------------------------------------------------ allocation-free totals */
/* The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory: code whose device memory is owned by
 * another allocator (a framework's caching allocator, a pool sized in
 * advance) or that must not let cudaMalloc synchronise the device between
 * its stream work.  It computes, in FP64 with a fixed reduction order,
 *   out[0] = sum_x sum_j f_j            out[1..3] = sum_x sum_j c_j f_j
 *   out[4] = sum_x |sum_j c_j f_j|^2 / (2 sum_j f_j)
 * for populations f given as q FP64 planes in rmrtlb_lattice_info order
 * (device memory of the current device, e.g. filled by
 * rmrtlb_get_populations).  Only RMRTLB_D2Q9, RMRTLB_D3Q19 and RMRTLB_D3Q27
 * are accepted; the axis-only lattices return RMRTLB_EINVAL.  f must hold
 * full populations (not deviations from a rest state); a node whose mass
 * sum_j f_j is exactly zero adds nothing to out[4].  For an unforced NSE
 * state these are the mass, momentum and kinetic energy that rmrtlb_stats
 * reports.
 *   out: host memory -> the totals are copied back and the call
 *        synchronises the stream before it returns; such a call cannot be
 *        captured into a CUDA graph, and during an active capture of the
 *        stream it returns RMRTLB_EINVAL without enqueueing anything.
 *        Device or managed memory of the current device -> the call is
 *        asynchronous: out is written in stream order, so synchronise the
 *        stream before reading a managed out on the host.
 * f or a device out on another GPU than the current one -> RMRTLB_EINVAL.
 * No solver and no workspace are needed: the reduction scratch is a fixed
 * array of (4096 * 8 + 8) doubles inside the library, present on every GPU
 * that loads it until the process exits.  At most RMRTLB_NOALLOC_MAX_NODES
 * nodes (nx*ny*nz) are accepted; larger grids return RMRTLB_ETOOBIG.  The
 * first call on a device looks the array up on that device and keeps its
 * address for the rest of the process; make that first call before any
 * stream capture, and do not call this entry point again on a device after
 * cudaDeviceReset (the kept address belonged to the destroyed context).  A
 * CUDA error left pending by earlier, unrelated work is returned as
 * RMRTLB_ECUDA before anything is launched, and is left pending for its
 * owner.  All calls share the array: calls whose kernels overlap on the GPU
 * (unordered streams) race and may return wrong totals; calls on one stream
 * are ordered.  Calls no cudaMalloc or cudaFree. */
#define RMRTLB_NOALLOC_MAX_NODES 67108864LL
int rmrtlb_population_totals_noalloc(int lattice, int nx, int ny, int nz,
                                     double dx, double dy, double dz, double dt,
                                     const double* f, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RMRTLB_H */
