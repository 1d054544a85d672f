/*
 * cmlbm -- cascaded central-moment lattice Boltzmann step with Galilean-invariant forcing,
 * as a C ABI over hand-written CUDA kernels for sm_103a (one GPU per handle).
 *
 * Method: K.N. Premnath and S. Banerjee, "Inertial frame independent forcing for discrete
 * velocity Boltzmann equation: implications for filtered turbulence simulation",
 * arXiv:1202.6074. Section and equation names below are the paper's.
 *
 * One step of the library (cmlbm_step) is, for every cell x:
 *   pull      g_i(x) = s_i(x - e_i)                    (standard streaming, Eq. cascadedstreaming1)
 *   moments   rho = sum g, rho u = sum g e + F/2        (Eqs. densitycalculation, velocitycalculation)
 *   central   kbar_a = sum g (e - u)^a                  (Sec. 7, transformed central moments)
 *   source    sigma_a by the exact hierarchical identity (Eq. centralmomentforceexactidentity2 with
 *             kappa = kbar + sigma/2, Eq. transformedcentralmoments)
 *   relax     post_a = kbar_a + omega_a (kappa^M_a - sigma_a/2 - kbar_a) + sigma_a
 *             (attractors Eq. centralmomenttransformed; procedure of Secs. 10-11)
 *   back      populations with the post-collision central moments (exact inverse, Sec. 9)
 *   store     s_i(x) <- post-collision population.
 * D3Q27, the Smagorinsky eddy viscosity, the boundaries and the storage formats are not in
 * the paper (it is written for D2Q9 and says the procedure extends to 3D, Secs. 2 and 15);
 * the readings used are stated at each field below.
 *
 * Conventions
 *   - Every function returns CMLBM_OK (0) or a negative CMLBM_ERR_* code; nothing throws.
 *     cmlbm_last_error() gives a message for the last failure on a handle.
 *   - Calls are asynchronous on the handle's stream, except cmlbm_reduce, cmlbm_create,
 *     cmlbm_destroy and calls with CMLBM_HOST buffers, which synchronise the stream.
 *   - Buffers passed in are owned by the caller and only borrowed for the call.
 *   - Test hook: with the environment variable CMLBM_TEST_ALLOC_LIMIT set to a byte count,
 *     every device allocation that grows with the grid (state, staging, force field, scratch)
 *     and is larger than that count fails with CMLBM_ERR_NOMEM without calling cudaMalloc.
 *   - Grid layout: cell (x, y, z) has linear index c = (z * ny + y) * nx + x; N = nx*ny*nz.
 *     Vector fields are [3][N] (component-major). Populations are [Q][N] (direction-major).
 *   - Direction order. D2Q9 (Sec. 2, Eq. velocityd2q9 with the order of the basis
 *     columns): 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *     D3Q27: i = 9*(ez+1) + 3*(ey+1) + (ex+1).
 *   - Rest weights w_i are the products of the 1D weights (1/6, 2/3, 1/6).
 *   - State format: s_i(x) holds the post-collision transformed population fbar of cell x
 *     encoded as d = fbar / w_i - 1 in the storage type (deviation from the rest weight,
 *     round-to-nearest-even on store). The library keeps two state buffers.
 */
#ifndef CMLBM_H
#define CMLBM_H

#include <stddef.h>

#if defined(__GNUC__)
#define CMLBM_API __attribute__((visibility("default")))
#else
#define CMLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define CMLBM_OK 0
#define CMLBM_ERR_INVALID (-1)      /* bad argument or configuration */
#define CMLBM_ERR_NOMEM (-2)        /* device or host allocation failed */
#define CMLBM_ERR_CUDA (-3)         /* a CUDA runtime call failed (message has the CUDA error) */
#define CMLBM_ERR_UNSUPPORTED (-4)  /* valid but not implemented for this configuration */
#define CMLBM_ERR_DIVERGED (-5)     /* a reduction found a non-finite value */

/* ---- enumerations ------------------------------------------------------------------ */
enum { CMLBM_D2Q9 = 0, CMLBM_D3Q27 = 1 };                          /* lattice */
enum { CMLBM_F64 = 0, CMLBM_F32 = 1, CMLBM_BF16 = 2, CMLBM_F16 = 3 }; /* state storage */
enum { CMLBM_PERIODIC = 0, CMLBM_BOUNCEBACK = 1, CMLBM_HALO = 2 };  /* per-axis boundary */
enum { CMLBM_DEVICE = 0, CMLBM_HOST = 1 };                         /* where a buffer lives */
enum { CMLBM_ATTRACTOR_MAXWELL = 0, CMLBM_ATTRACTOR_FACTORIZED = 1 };
enum { CMLBM_KERNEL_AUTO = 0, CMLBM_KERNEL_DIRECT = 1, CMLBM_KERNEL_TMA = 2, CMLBM_KERNEL_PAIR = 3,
       CMLBM_KERNEL_PAIR_TWO_STEPS = 4 };

typedef struct cmlbm cmlbm_t;

/*
 * Configuration. Fill with cmlbm_config_default() and override.
 *   lattice, nx, ny, nz   D2Q9 needs nz == 1. Each size >= 1, N < 2^31 and Q * N < 2^32.
 *   storage               arithmetic is FP64 for CMLBM_F64 storage and FP32 otherwise.
 *   bc[3]                 per axis (x, y, z). Bounce-back puts half-way walls outside the
 *                         first and last cells of that axis (paper silent on boundaries):
 *                         g_i(x) = s_ibar(x) + 2 w_i rho_w (e_i . u_w) / c_s^2, rho_w = 1, u_w the
 *                         crossed wall's velocity (the mean of both walls on an edge link).
 *                         CMLBM_HALO (z axis of D3Q27 only): the handle is one z-slab of a larger
 *                         domain (see "slab decomposition" below); each state buffer carries one
 *                         ghost plane below z = 0 and one above z = nz - 1, and z does not wrap.
 *   wall_velocity[a][s]   velocity of the wall on axis a, side s (0 = below index 0, 1 = above n-1).
 *   tau                   shear relaxation time: omega_nu = 1/tau, nu = c_s^2 (tau - 1/2)
 *                         (Sec. 10, text after Eq. collisionkernelg8). Must satisfy tau > 1/2.
 *   omega_bulk            rate of the trace of the second-order central moments (omega_3 of
 *                         the paper); 0 = follow the (effective) shear rate.
 *   omega_3, omega_4      rates of the third-order and of the fourth- and higher-order central
 *                         moments (0 < omega < 2, Sec. 10).
 *   smagorinsky_cs        Smagorinsky constant C_s; 0 disables the eddy viscosity. Reading
 *                         (paper silent on the model; frame invariance required by Sec. 1):
 *                         Pi = kappa_ij - c_s^2 rho delta_ij from second-order central moments,
 *                         Q = |Pi|, tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 Q / rho)) / 2.
 *                         With FP32 arithmetic (FP32 and 16-bit storage) the two square roots
 *                         and 1 / tau_eff use the hardware approximations (within a few ulp);
 *                         FP64 storage uses the rounded operations.
 *   van_driest_aplus      A+ of the damping C = C_s (1 - exp(-y+/A+)); 0 disables. Needs y walls.
 *   van_driest_utau_over_nu  u_tau / nu_0 so that y+ = y_wall * u_tau / nu_0, y_wall = distance to
 *                         the nearest y wall (j + 1/2 or ny - 1/2 - j).
 *   attractor             CMLBM_ATTRACTOR_MAXWELL (Eq. centralmomenttransformed) or
 *                         CMLBM_ATTRACTOR_FACTORIZED (Sec. 13, Eq. factorxxyyfinal).
 *   reduced_compressibility  1 = momentum rho0 u = sum fbar e + F/2 (Sec. 12).
 *   rho0                  reference density of the reduced-compressibility form.
 *   stream                cudaStream_t to launch on; NULL = the legacy default stream.
 *   device                CUDA device ordinal the handle lives on.
 *   kernel                step kernel: CMLBM_KERNEL_AUTO (the fastest measured that the
 *                         configuration allows: two cells per thread, else one cell per
 *                         thread), CMLBM_KERNEL_DIRECT (one cell per thread),
 *                         CMLBM_KERNEL_PAIR (two cells of a row per thread in packed FP32
 *                         arithmetic), CMLBM_KERNEL_PAIR_TWO_STEPS (the PAIR kernel scheduled two
 *                         steps per pass: z-planes in groups of 8, the intermediate state in a
 *                         ring of 12 planes meant to stay in L2; FP32 storage, no slab,
 *                         nz >= 16; bitwise the same results, measured slower than PAIR on
 *                         GB300), or CMLBM_KERNEL_TMA (rows staged in shared memory by TMA).
 *                         PAIR covers D3Q27 with FP32 / BF16 / FP16 storage, periodic x and nx a
 *                         multiple of 64, in every collision form (PAIR_TWO_STEPS: the Maxwellian
 *                         attractor and standard compressibility only);
 *                         TMA covers D3Q27 with FP32 / BF16 / FP16 storage, nx a multiple of 128,
 *                         the Maxwellian attractor, standard compressibility, and no slab. An
 *                         explicit choice the configuration cannot use fails with
 *                         CMLBM_ERR_UNSUPPORTED.
 */
typedef struct {
    int lattice;
    int nx, ny, nz;
    int storage;
    int bc[3];
    double wall_velocity[3][2][3];
    double tau;
    double omega_bulk;
    double omega_3;
    double omega_4;
    double smagorinsky_cs;
    double van_driest_aplus;
    double van_driest_utau_over_nu;
    int attractor;
    int reduced_compressibility;
    double rho0;
    void* stream;
    int device;
    int kernel;
} cmlbm_config;

/* Defaults: D3Q27, 32^3, FP32, periodic, tau = 0.8, omega_bulk = 0, omega_3 = omega_4 = 1,
 * no eddy viscosity, Maxwellian attractor, rho0 = 1, default stream, device 0. */
CMLBM_API int cmlbm_config_default(cmlbm_config* cfg);

/* Validate cfg, allocate two state buffers of cmlbm_state_bytes() each on cfg->device and
 * initialise the rest state (rho = 1, u = 0, F = 0). *out receives the handle.
 * Errors: CMLBM_ERR_INVALID (bad sizes, tau <= 1/2, D2Q9 with nz != 1, van Driest without
 * y walls, an unknown kernel), CMLBM_ERR_UNSUPPORTED (an explicit kernel choice the
 * configuration cannot use), CMLBM_ERR_NOMEM, CMLBM_ERR_CUDA. On error *out is NULL. */
CMLBM_API int cmlbm_create(const cmlbm_config* cfg, cmlbm_t** out);

/* Release all device memory of the handle. NULL-safe. Synchronises the handle's stream. */
CMLBM_API void cmlbm_destroy(cmlbm_t* h);

/* Message of the last failed call on h, or of the last failed cmlbm_create on this thread
 * when h is NULL. The string lives until the next failing call. */
CMLBM_API const char* cmlbm_last_error(const cmlbm_t* h);

/* Replace the stream the handle launches on (cudaStream_t, NULL = default stream). */
CMLBM_API int cmlbm_set_stream(cmlbm_t* h, void* stream);

/* Set the body force (paper: F in Eqs. cascadedLBE1 - velocitycalculation). uniform[3] is
 * added to every cell; field (FP64, [3][N], on `where`) replaces it when non-NULL and is
 * copied into the handle in the arithmetic precision (FP64 or FP32). NULL uniform = 0. */
CMLBM_API int cmlbm_set_force(cmlbm_t* h, const double uniform[3], const double* field, int where);

/* Initialise the state so that the next pull returns fbar = f^M(rho, u) - S/2 with the
 * current force, S evaluated at the Maxwellian moments (paper silent on initialisation;
 * the special case noted under Eq. exactidentitycomponents). rho [N] and u [3][N] are FP64
 * on `where`; rho NULL means 1, u NULL means 0. With CMLBM_HOST, page-locked buffers that the
 * CUDA runtime maps for the device (cudaHostAlloc, cudaMallocHost) are read in place by the
 * init kernel; other host memory is staged through a device buffer. */
CMLBM_API int cmlbm_init(cmlbm_t* h, const double* rho, const double* u, int where);

/* Advance nsteps stream-and-collide steps (nsteps >= 0): the pull of Eq. cascadedstreaming1
 * followed by the collision of Sec. 10, fused in one kernel launch per step, asynchronous on the
 * handle's stream. Pairs of steps are replayed as a CUDA graph (captured once per buffer parity
 * on a private stream, dropped when the force changes), so a call of many steps costs one graph
 * launch per two steps; a failed capture falls back to plain launches for the handle's life. */
CMLBM_API int cmlbm_step(cmlbm_t* h, int nsteps);

/* One step from the state buffer src into dst (device pointers of cmlbm_state_bytes() each,
 * in the handle's layout, src != dst), with the handle's configuration and force. Used for
 * checkpointed recomputation; the handle's own state is untouched. Buffers need the alignment
 * of one storage element; buffers aligned to two elements (any cudaMalloc allocation) let the
 * two-cells-per-thread kernel pair adjacent cells, which gives the same bits faster. */
CMLBM_API int cmlbm_step_buffers(cmlbm_t* h, const void* src, void* dst);

/* Density [N] and velocity [3][N] (FP64) of the current pre-collision field (pull of the
 * stored state): Eqs. densitycalculation and velocitycalculation (reduced-compressibility
 * form: u = (sum fbar e + F/2) / rho0). Either pointer may be NULL. With CMLBM_HOST,
 * page-locked mapped buffers are written in place by the moments kernel (other host memory
 * through a device staging buffer); the call returns when the values are in host memory. */
CMLBM_API int cmlbm_moments(cmlbm_t* h, double* rho, double* u, int where);

/* Same as cmlbm_moments for an arbitrary state buffer (device, handle layout). */
CMLBM_API int cmlbm_moments_of(cmlbm_t* h, const void* state, double* rho, double* u);

/* FP64 reductions of the current field: out = {sum rho, sum j_x, sum j_y, sum j_z,
 * sum rho |u|^2 / 2} (host array, synchronous, deterministic order), where j = sum fbar e + F/2
 * is the momentum of Eq. velocitycalculation (rho u; rho0 u in the reduced-compressibility form of
 * Sec. 12, whose velocity is u = j / rho0). Each cell's values are computed in the arithmetic
 * precision and summed in FP64. Returns CMLBM_ERR_DIVERGED if any of the five is not finite (a
 * NaN or infinity anywhere in the field reaches the sums), and CMLBM_ERR_CUDA if a TMA-staged step
 * since the last check gave up on a bounded pipeline wait (its output is then invalid).
 *
 * TMA-staged steps report a pipeline wait that gave up through a device flag. Its value is copied
 * to the host after every cmlbm_step / cmlbm_step_buffers call, asynchronously; every call that
 * returns results (cmlbm_step, cmlbm_step_buffers, cmlbm_moments, cmlbm_moments_of,
 * cmlbm_get_state, cmlbm_reduce) checks it on entry, and the synchronising ones (cmlbm_reduce and
 * the CMLBM_HOST forms of cmlbm_moments and cmlbm_get_state) check it again once the stream is
 * drained. A failure is reported once, by CMLBM_ERR_CUDA, and the flag is then cleared. */
CMLBM_API int cmlbm_reduce(cmlbm_t* h, double out[5]);

/* Bytes of one state buffer: Q * N * storage size, or Q * nx * ny * (nz + 2) * storage size
 * with bc[2] = CMLBM_HALO (the ghost planes are part of the state). */
CMLBM_API size_t cmlbm_state_bytes(const cmlbm_t* h);

/* Copy the current state out of / into the handle (raw storage format, bytes must equal
 * cmlbm_state_bytes). */
CMLBM_API int cmlbm_get_state(cmlbm_t* h, void* dst, size_t bytes, int where);
CMLBM_API int cmlbm_set_state(cmlbm_t* h, const void* src, size_t bytes, int where);

/* ---- turbulence as forcing (Sec. 14, filtered kinetic equation) -------------------------- *
 * The unresolved stresses act as the body force F = rho a', a'_i = -d_j (u'_i u'_j), with the
 * resolved momentum rho0 u = sum fbar e + rho a' / 2 (Eq. resolvedvelocitycalculation; configure
 * reduced_compressibility = 1 and, as the paper suggests, the factorized attractor). Closure
 * (paper: any conventional macroscopic model): Smagorinsky, u'_i u'_j (deviatoric) = -2 nu_t S_ij,
 * nu_t = cs^2 |S|, |S| = sqrt(2 S:S), S from second-order central differences of the resolved
 * velocity of the current field (computed with the force in place), lattice spacing 1.
 * cmlbm_turbulence_force sets the handle's force field to rho a' plus the uniform force last
 * given to cmlbm_set_force; cmlbm_step_filtered repeats {turbulence_force; step} nsteps times.
 * Periodic boundaries only (CMLBM_ERR_UNSUPPORTED otherwise). Allocates 13 N arithmetic values
 * of scratch and force field on first use. */
CMLBM_API int cmlbm_turbulence_force(cmlbm_t* h, double cs);
CMLBM_API int cmlbm_step_filtered(cmlbm_t* h, int nsteps, double cs);

/* ---- adjoint (reverse mode of cmlbm_step_buffers; paper silent) ---------------------- *
 * Adjoint state lambda is [Q][N] in the arithmetic precision (FP64 for F64 storage, FP32
 * otherwise) and holds dL/ds for the post-collision populations s (not the encoded d).
 * dLdF is an FP64 [3][N] accumulator. Supported for F64 and F32 storage, Maxwellian
 * attractor, standard compressibility, without eddy viscosity; else CMLBM_ERR_UNSUPPORTED. */

/* Terminal adjoint of a loss on the velocity of state s_T: given dL/du ([3][N] FP64,
 * device) and optionally dL/drho ([N], NULL = 0), writes lambda_T = dL/ds_T and adds the
 * direct force term (u depends on F through F/2) into dLdF. */
CMLBM_API int cmlbm_adjoint_terminal(cmlbm_t* h, const void* state, const double* dLdu, const double* dLdrho,
                           void* lambda, double* dLdF);

/* One step back: state is s_t (the input of the step s_t -> s_{t+1}), lambda_in = dL/ds_{t+1},
 * lambda_out = dL/ds_t (must not alias lambda_in); adds (dC/dF)^T lambda_in into dLdF. */
CMLBM_API int cmlbm_step_adjoint(cmlbm_t* h, const void* state, const void* lambda_in, void* lambda_out, double* dLdF);

/* cmlbm_step_adjoint with the force gradient of the step, (dC/dF)^T lambda_in, added into a
 * segment accumulator seg ([3][N] device array in the arithmetic precision: FP32 for F32
 * storage, FP64 for F64) instead of into dLdF. With fold != 0, seg with this step's term is then
 * added into the FP64 dLdF and seg is set to zero. A reverse sweep over a checkpoint segment
 * passes fold = 1 on its last call (the segment's first step): the per-step traffic of the
 * accumulator is then 2 x 12 bytes per cell at FP32 instead of 2 x 24, and the sum over
 * segments stays in FP64. seg must be zero before the first call of a segment (cudaMemset, or
 * a previous fold). Errors as for cmlbm_step_adjoint, and CMLBM_ERR_INVALID for a NULL seg. */
CMLBM_API int cmlbm_step_adjoint_segment(cmlbm_t* h, const void* state, const void* lambda_in, void* lambda_out,
                                         void* seg, double* dLdF, int fold);

/* ---- slab decomposition along z (no counterpart in the paper) -------------------------- *
 * A periodic-in-z D3Q27 domain split into z-slabs, one handle per slab, each created with
 * bc[2] = CMLBM_HALO and nz = its own number of planes. The streaming step (Eq.
 * cascadedstreaming1) pulls s_i(x - e_i): the only values a slab reads from outside itself are
 * those of the 9 directions with e_z = +1 from the plane just below it and of the 9 with
 * e_z = -1 from the plane just above. Each state buffer is laid out [Q][nz + 2][ny][nx] with
 * those two ghost planes at z = -1 and z = nz; steps, moments and reductions cover the nz own
 * planes and read the ghosts. After every step the caller refreshes the ghosts from the
 * neighbours (the slab below is the periodic predecessor, the slab above the successor):
 *     top    = pack(CMLBM_FACE_TOP)     -> unpack(CMLBM_FACE_BOTTOM) on the slab above
 *     bottom = pack(CMLBM_FACE_BOTTOM)  -> unpack(CMLBM_FACE_TOP)    on the slab below
 * cmlbm_init writes valid ghosts itself (the inverse pull of the slab's own cells), so the first
 * step needs no exchange. A one-slab domain is its own neighbour on both sides. Moving and
 * resting walls on x and y, force fields, eddy viscosity and all collision forms work as in a
 * single domain; the TMA step, the adjoint and turbulence forcing return
 * CMLBM_ERR_UNSUPPORTED on a slab handle. */
enum { CMLBM_FACE_BOTTOM = 0, CMLBM_FACE_TOP = 1 };

/* One step like cmlbm_step(h, 1), split so that a slab's face exchange can overlap its update:
 * the first and last planes (z = 0 and nz - 1, the only ones whose pull reads the ghost planes,
 * and the only ones the next face messages come from) are launched on the handle's stream, the
 * interior planes 1 .. nz - 2 on a stream of the library's own. A pack issued on the handle's
 * stream right after this call waits only for the two boundary planes, and the unpacks write
 * ghost planes that the interior launch does not read, so the exchange proceeds while the
 * interior runs. The next split step orders its boundary planes after this interior (they pull
 * from planes 1 and nz - 2) and its interior after everything issued on the handle's stream
 * before it; every other call that reads or writes the state or the force (cmlbm_step,
 * cmlbm_moments, cmlbm_reduce, cmlbm_get_state, ...) first orders the handle's stream after the
 * interior. Same results, bit for bit, as cmlbm_step(h, 1). Any handle with the direct or
 * two-cells-per-thread kernel (CMLBM_ERR_UNSUPPORTED for the TMA-staged and two-steps kernels);
 * meant for slabs. The private stream and two events are created on the first call.
 * parts = CMLBM_SPLIT_BOTH issues both parts. CMLBM_SPLIT_BOUNDARY and then CMLBM_SPLIT_INTERIOR
 * issue them in two calls, so that a driver of several slabs on one GPU can issue every slab's
 * boundary planes before any interior: a kernel issued after a large one waits for the large
 * one's blocks to be dispatched. The state becomes the new one (for packs, moments, ...) once
 * the interior part is issued; the two parts of a step must alternate (CMLBM_ERR_INVALID
 * otherwise). The interior stream has the lowest priority: issue the split steps and the face
 * exchange on a stream of higher priority (cudaStreamCreateWithPriority, cmlbm_set_stream), or
 * the small boundary launches and copies wait behind the interior's blocks and nothing overlaps
 * (measured on one GB300 with two slabs of a 256^3 box: 0.99 of one domain's rate with a
 * high-priority stream, 0.91 without). */
enum { CMLBM_SPLIT_BOUNDARY = 1, CMLBM_SPLIT_INTERIOR = 2, CMLBM_SPLIT_BOTH = 3 };
CMLBM_API int cmlbm_step_split(cmlbm_t* h, int parts);

/* Bytes of one face message: 9 * nx * ny values in the storage format. */
CMLBM_API size_t cmlbm_halo_bytes(const cmlbm_t* h);

/* Copy the 9 populations that leave the slab through `face` out of the current state:
 * CMLBM_FACE_TOP = directions with e_z = +1 of plane nz - 1, CMLBM_FACE_BOTTOM = e_z = -1 of
 * plane 0. out holds [9][ny][nx] values in the storage format, directions in increasing
 * lexicographic order (index 9 (e_z + 1) + 3 (e_y + 1) + (e_x + 1)); where = CMLBM_DEVICE
 * (asynchronous on the handle's stream) or CMLBM_HOST (returns when the copy has landed).
 * CMLBM_ERR_INVALID for a bad face, NULL out, or a handle without CMLBM_HALO on z. */
CMLBM_API int cmlbm_halo_pack(cmlbm_t* h, int face, void* out, int where);

/* Write a neighbour's face message into a ghost plane of the current state:
 * CMLBM_FACE_BOTTOM = the ghost below (takes the slab below's TOP message), CMLBM_FACE_TOP =
 * the ghost above (takes the slab above's BOTTOM message). Layout and `where` as for
 * cmlbm_halo_pack; a host buffer may be reused when the call returns. */
CMLBM_API int cmlbm_halo_unpack(cmlbm_t* h, int face, const void* in, int where);

/* Kernel launches issued by the handle so far (for benchmark accounting). */
CMLBM_API long long cmlbm_launch_count(const cmlbm_t* h);

/* The step kernel the handle runs: CMLBM_KERNEL_DIRECT, CMLBM_KERNEL_PAIR,
 * CMLBM_KERNEL_PAIR_TWO_STEPS or CMLBM_KERNEL_TMA (what CMLBM_KERNEL_AUTO resolved to);
 * CMLBM_ERR_INVALID for a NULL handle. */
CMLBM_API int cmlbm_step_kernel(const cmlbm_t* h);

/* ---- allocation-free reduction (no counterpart in the paper) --------------------------- *
 * The FP64 reductions of cmlbm_reduce for callers that cannot allocate device memory: a host
 * whose device memory is all handed out up front to another allocator (a framework's memory
 * pool, where an outside cudaMalloc fails or fragments the pool), a loop with a fixed memory
 * budget that must not grow its footprint while it runs, or a tool that must not create a
 * handle (cmlbm_create allocates two state buffers).
 * No handle and no allocation: the caller passes the configuration, a state buffer in the
 * library's layout and storage format (device, Q*N elements), the force (uniform[3] added
 * everywhere, NULL = 0; force_field = device [3][N] array in the arithmetic type -- double for
 * CMLBM_F64 storage, float otherwise -- or NULL), and out, a device array of 5 doubles that
 * receives {sum rho, sum j_x, sum j_y, sum j_z, sum rho |u|^2 / 2} as cmlbm_reduce defines them.
 * Launches asynchronously on cfg->stream (device cfg->device); the caller synchronises.
 * Scratch: the per-block partial sums live in one file-scope device array of 16384 x 5
 * doubles (640 KiB on every GPU that loads the library, kept until the process exits), so
 * grids are limited to nx*ny*nz <= 16,777,216 cells; larger grids return CMLBM_ERR_INVALID
 * before anything is launched. Every block overwrites its own partials, so nothing needs
 * clearing between calls, but all calls share the array: calls that overlap on the GPU
 * (different streams, or host threads racing) corrupt each other's sums. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and keeps it for the life of the process; make that first call before any stream
 * capture begins. A cudaDeviceReset of that device unloads the library's device code and may move
 * the array, so the kept address is no longer valid: do not call this entry point on a device
 * after resetting it.
 * Errors: CMLBM_ERR_INVALID (NULL arguments, bad configuration, grid over the limit),
 * CMLBM_ERR_CUDA (symbol lookup or launch failure). */
CMLBM_API int cmlbm_reduce_noalloc(const cmlbm_config* cfg, const void* state, const double uniform_force[3],
                                   const void* force_field, double* out);

#ifdef __cplusplus
}
#endif

#endif /* CMLBM_H */
