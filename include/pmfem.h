/*
 * pmfem.h -- C-ABI of the periodic micromagnetic FEM effective-field library (libpmfem.so).
 *
 * What it computes (Ai, Duan, Lomakin, "Periodic micromagnetic finite element method"):
 *   H_eff = H_ex + H_ms + H_ap                                   (Eq. 3, no anisotropy)
 *   H_ex  : periodized P1 Laplacian, Eqs. 7-12
 *   H_ms  : charges (Eq. 14a) -> projection onto a uniform grid (BAIM step 1) -> FFT
 *           convolution with the periodic Green's function of Eq. 15 (step 2) ->
 *           interpolation (step 3) -> near-field precorrection (step 4, Eq. 14c) ->
 *           periodized gradient (Eq. 14d)
 *   LLG   : Eq. 2 / Eq. 6, integrated by classical RK4 with renormalisation.
 * Units are SI (metres, A/m, J/m, seconds); magnetisation arguments are unit vectors m
 * (M = Ms m is applied inside).
 *
 * Conventions shared by every call
 *   - Every function returns int: 0 on success, a negative PMFEM_E* code on failure.
 *     pmfem_last_error(h) gives a message for the last failing call on that handle.
 *   - Handles are opaque.  The library owns all device memory it allocates; the caller
 *     owns every buffer it passes in.  Host arrays passed in are copied before the call
 *     returns and may be freed afterwards.
 *   - "device" pointers are CUDA device (or managed) addresses; "host" pointers are CPU
 *     addresses (pinned memory makes the host-buffer calls faster but is not required).
 *   - stream is a cudaStream_t passed as void*; NULL selects the library's own stream,
 *     which is a blocking stream (ordered with the legacy default stream).
 *     Calls that take a stream enqueue work and return without synchronising, except
 *     where stated.
 *   - Unknown ordering: the N' unknowns are the ancestors of the periodic pairing
 *     (Sec. 2.2), numbered by increasing original node index; pmfem_lca_map gives the
 *     unknown of every original node.  Field/state arrays are N' x 3, row-major.
 *   - Precision (pmfem_set_precision) fixes the element type T of field/state buffers:
 *     PMFEM_FP64 -> double; PMFEM_FP32 and PMFEM_BF16SPLIT -> float.
 *   - Set-up (create_mesh, set_aim, set_periodicity) runs on the host and does not touch
 *     the GPU; device buffers are allocated on the first call that needs them.
 *   - A handle (and a batch) is used by one host thread at a time: its scratch buffers, its
 *     second stream and its fork/join events are per handle, so two calls on one handle
 *     must not overlap.  Different handles are independent (pmfem_field_noalloc excepted,
 *     see there).
 */
#ifndef PMFEM_H
#define PMFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmfem_state* pmfem_t;

/* status codes */
#define PMFEM_OK          0
#define PMFEM_EINVAL     -1   /* bad argument (size, NULL, out-of-range value)          */
#define PMFEM_ENOMEM     -2   /* host or device allocation failed                       */
#define PMFEM_ECUDA      -3   /* a CUDA runtime call failed (no GPU, launch failure)    */
#define PMFEM_EMESH      -4   /* invalid mesh: bad index, degenerate tetrahedron,
                                 unpaired node on a touching periodic face               */
#define PMFEM_ENONFINITE -5   /* NaN/Inf met in an input or a result (device check)      */
#define PMFEM_ETIMEOUT   -6   /* a bounded device wait ran out                          */
#define PMFEM_ESTATE     -7   /* call out of order (e.g. field before set_periodicity)  */
#define PMFEM_ENOCONV    -8   /* an iterative solve (Newton) did not converge            */

/* precision modes */
#define PMFEM_FP64      0
#define PMFEM_FP32      1
#define PMFEM_BF16SPLIT 2     /* split precision: the operators chosen by
                                 pmfem_set_bf16_operators are stored in bfloat16, all
                                 others and every vector and grid buffer in FP32; all
                                 arithmetic and accumulation in FP32                    */

/* operator bitmask for pmfem_set_bf16_operators */
#define PMFEM_BF16_PRECORRECTION 1   /* point precorrection C (BAIM step 4)                 */
#define PMFEM_BF16_PROJECTION    2   /* Lagrange weights of the projection (step 1)         */
#define PMFEM_BF16_CHARGES       4   /* W^q of Eq. 14a and the near-element E of Eq. 14c    */
#define PMFEM_BF16_GRADIENT      8   /* -V^-1 (W^q)^T of Eq. 14d                            */
#define PMFEM_BF16_EXCHANGE     16   /* periodized Laplacian of Eq. 8                       */

/* field component bitmask for pmfem_field */
#define PMFEM_EX 1      /* exchange (Eqs. 7-12)                                                */
#define PMFEM_MS 2      /* magnetostatic (Eq. 14)                                              */
#define PMFEM_AP 4      /* applied field                                                        */
#define PMFEM_AN 8      /* anisotropy (pmfem_set_anisotropy; zero when none is set)            */
#define PMFEM_ALL 15

/* Library version string and the last error message of a handle (never NULL). */
const char* pmfem_version(void);
const char* pmfem_last_error(pmfem_t h);

/*
 * Create a mesh handle (Sec. 2.2 discrete formulation, P1 tetrahedra, Eq. 4).
 *   xyz   host, N x 3 doubles, node coordinates in metres; N <= 2^30 (else EINVAL)
 *   tets  host, T x 4 int32, node indices in [0, N); negatively oriented tetrahedra
 *         are re-oriented, tetrahedra with 6|V| <= 1e-12 * (longest edge)^3 -> EMESH
 *   Ms    saturation magnetisation [A/m] (> 0); A exchange stiffness [J/m] (>= 0);
 *   alpha Gilbert damping (>= 0).
 * The handle starts non-periodic with default AIM settings; *out is NULL on failure.
 */
int pmfem_create_mesh(pmfem_t* out, const double* xyz, int64_t N, const int32_t* tets, int64_t T,
                      double Ms, double A, double alpha);

/*
 * AIM grid and near-zone settings (Sec. 3.2, Eq. 16, Eq. 17).  Call before
 * pmfem_set_periodicity; 0 selects the default for each argument.
 *   Nx, Ny, Nz   grid points per axis.  A periodic axis uses Delta = L / N and an FFT of
 *                length N; a non-periodic axis uses Delta = D / (N - 1 - 2m) with
 *                m = ceil((p+1)/2) halo cells and an FFT of length 2N.  Every FFT length
 *                must be a power of two between 4 and 1024.  Default: about 2 grid points
 *                per mean edge length, rounded up to a power of two.
 *   order_p      Lagrange stencil order, 2..5 ((p+1)^3 points per node); default 3.
 *   near_boxes   Chebyshev radius in grid cells of the point-pair precorrection; default 3.
 *   near_elem_factor  radius of the exact element correction in mean edge lengths; 0 keeps
 *                only elements touching the observer node (default 0).
 */
int pmfem_set_aim(pmfem_t h, int Nx, int Ny, int Nz, int order_p, int near_boxes, double near_elem_factor);

/*
 * Periods L1, L2, L3 [m] along x, y, z (Eq. 1 / Eq. 5): L > 0 makes the axis periodic,
 * 0 leaves it open; any subset of axes may be periodic.  Runs the whole host set-up in
 * FP64: PBC pairing and LCA (tolerance 1e-9 min L), the protruding fold of Eq. 18, the
 * periodized operators, the grid, the PGF spectrum (Eq. 15, Ewald-type sums) and the
 * precorrection matrices.  EMESH when a node on a touching periodic face has no partner.
 * May be called again (with new periods) to redo the set-up.
 */
int pmfem_set_periodicity(pmfem_t h, double L1, double L2, double L3);

/*
 * Local terms of Eq. 3 beyond exchange (the paper's granular example, Sec. 4.4: grains with
 * their own crystal axes and a reduced exchange across grain boundaries).
 *
 * pmfem_set_exchange_per_tet: exchange stiffness of every tetrahedron, A_tet host T doubles
 * [J/m] (>= 0), in place of the uniform A of pmfem_create_mesh: the exchange operator becomes
 * -(2/(mu0 Ms)) V^-1 K_A with (K_A)_nk = sum_e A_e V_e grad(phi_n).grad(phi_k) (Eq. 8 with A
 * inside the element sum; tetrahedra of a grain-boundary layer carry the inter-grain A_iex).
 * NULL returns to the uniform A.  Takes effect at the next pmfem_set_periodicity.
 *
 * pmfem_set_anisotropy: the grain of every tetrahedron (tet_grain, host T int32 in
 * [0, n_grains)) and per grain its crystal axes (axes, host n_grains x 9 doubles: three unit
 * rows a1, a2, a3), cubic constant K1 [J/m^3] (host n_grains or NULL) and uniaxial constant Ku
 * [J/m^3] with axis u (host n_grains and n_grains x 3, or both NULL).  With a_i = m . a_i the
 * fields are -(2 K1/(mu0 Ms)) sum_i a_i (a_j^2 + a_k^2) a_i and (2 Ku/(mu0 Ms)) (m.u) u; the
 * nodal field is the volume-weighted mean over the grains of the tetrahedra at the node (the
 * energy lumped to the nodes).  It enters pmfem_field under PMFEM_AN (and PMFEM_ALL), the RK4
 * and implicit steps (the implicit step's Jacobian leaves it out: its Newton iteration becomes
 * a quasi-Newton iteration for it), in the field kernel's epilogue.  Batches ignore it.
 * tet_grain NULL removes it.  An accepted call drops the handle's device data (the state m
 * included); EINVAL, with the handle unchanged, for grains out of range, axes that are not unit
 * rows, Ku without u, neither K1 nor Ku, or non-finite constants.
 */
int pmfem_set_exchange_per_tet(pmfem_t h, const double* A_tet);
int pmfem_set_anisotropy(pmfem_t h, const int32_t* tet_grain, int n_grains, const double* K1, const double* axes,
                         const double* Ku, const double* u);

/*
 * Where pmfem_set_periodicity evaluates the FP64 set-up arithmetic that grows with the mesh
 * and the grid (the paper does it once, in preprocessing, Sec. 4): use_gpu 0 (default) on
 * the host's threads; 1 as CUDA kernels on the current device, in FP64, for the PGF spectrum
 * (Eq. 15 by Ewald-type sums on the grid of Eq. 16, and its transform), the exact near-element
 * integrals of Eq. 14c and the point precorrection of BAIM step 4 (Sec. 3.2).  Both evaluate
 * the same formulas in the same order and agree to the rounding of the two sides' math
 * libraries.  With 1, pmfem_set_periodicity allocates temporary device memory (freed before it
 * returns), synchronises the device, and fails with ECUDA (no GPU) or ENOMEM.  Pairing, the
 * local operators, the grid and the placement search stay on the host.  Takes effect at the
 * next pmfem_set_periodicity.  EINVAL for other values.
 */
int pmfem_set_setup_device(pmfem_t h, int use_gpu);

/*
 * Device layout tuning (no paper counterpart; it changes speed, not results beyond
 * rounding).  Unknowns are stored sorted by grid box in tiles of tile_y box rows x tile_z
 * box planes (x fastest); precorrection rows may be sorted by length inside windows of
 * sort_window rows; column indices are stored as deltas to a per-row base, modulo N', in
 * 16 bits when every delta fits (col_bits 0 or 16) or in 32 bits (col_bits 32).  0 selects the defaults (8, 4, 1024,
 * 16-bit when possible).  Takes effect at the next device upload; may come before or after pmfem_set_periodicity.
 */
int pmfem_set_layout(pmfem_t h, int tile_y, int tile_z, int sort_window, int col_bits);

int pmfem_set_precision(pmfem_t h, int mode);                       /* PMFEM_FP64 | FP32 | BF16SPLIT */

/*
 * Operators stored in bfloat16 under PMFEM_BF16SPLIT (bitmask of PMFEM_BF16_*; the method
 * itself is precision-agnostic, Sec. 4 runs it in single precision).  Values are rounded
 * once from the FP64 set-up to the nearest bfloat16 (ties to even) and widened exactly to
 * FP32 in the kernels, so each chosen operator carries a relative error of at most 2^-9 per
 * entry and moves half the bytes.  Default PMFEM_BF16_PRECORRECTION | PMFEM_BF16_PROJECTION
 * | PMFEM_BF16_GRADIENT.  The charge operator (Eq. 14a) and the exchange operator (Eq. 8)
 * stay in FP32 by default: both act on m itself, whose neighbouring values nearly cancel
 * (charges are a divergence, exchange a Laplacian), so a 2^-9 error per entry grows into
 * an error of a few 1e-3 (magnetostatic field) and a few 1e-2 (exchange field) on a
 * smooth m.  Takes effect at the next device upload (a change under an uploaded
 * BF16-split device drops its data, the state m included).  EINVAL for bits outside the
 * five flags.
 */
int pmfem_set_bf16_operators(pmfem_t h, int mask);
int pmfem_set_applied_field(pmfem_t h, double Hx, double Hy, double Hz);   /* A/m, uniform       */

/* Number of unknowns N' (Sec. 2.2) and the node -> unknown map (host, N int32). */
int pmfem_num_unknowns(pmfem_t h, int64_t* n_unknowns);
int pmfem_lca_map(pmfem_t h, int32_t* host_out);

/*
 * One effective-field evaluation (Eq. 3).
 *   m      device, N' x 3 T, unit vectors (read only)
 *   H      device, N' x 3 T, written in A/m (may not alias m)
 *   components  bitmask of PMFEM_EX | PMFEM_MS | PMFEM_AP
 * Enqueued on stream; a non-finite m sets a device flag reported as ENONFINITE by the
 * next pmfem_sync.  In FP32 and BF16-split, the precorrection part of the magnetostatic
 * field runs on a second stream of the handle, forked from stream after the charges and
 * joined back into it before the stencil pass (CUDA events): the evaluation stays ordered on
 * stream as a whole, and a graph capture on stream captures both branches.
 */
int pmfem_field(pmfem_t h, const void* m, void* H, int components, void* stream);

/* Same as pmfem_field with host buffers (N' x 3 T each): copies in, evaluates, copies
 * out and synchronises the stream before returning. */
int pmfem_field_host(pmfem_t h, const void* m_host, void* H_host, int components, void* stream);

/*
 * pmfem_field without any allocation (the paper has no counterpart; this is a service for
 * callers that must not allocate device memory when they ask for a field: real-time loops
 * that forbid allocator calls, or hosts whose device memory belongs to a pooling
 * allocator).  Same arguments and same result as pmfem_field; all scratch of the
 * evaluation lives in one fixed 64 MiB device array compiled into the library.  The array
 * is reserved on a device when the library's device code is loaded there (with CUDA's lazy
 * module loading, at the latest when a handle's device data are first built on it) and is
 * kept until the process exits.  The call allocates nothing itself:
 *   - the handle's operators must already be on the device at the current precision (one
 *     earlier pmfem_field or pmfem_set_m call); otherwise ESTATE.  That earlier call also
 *     looks up the array's device address (cudaGetSymbolAddress, in the context then
 *     current), so pmfem_field_noalloc itself makes no CUDA call but its kernel launches;
 *   - a mesh and grid whose scratch exceeds 64 MiB give EINVAL (use pmfem_field);
 *   - every call on a device shares the one array: calls that overlap on the GPU (other
 *     streams, other handles) race and must be serialised by the caller.  Nothing in the
 *     array needs to start at zero; it keeps whatever the last call left.
 */
int pmfem_field_noalloc(pmfem_t h, const void* m, void* H, int components, void* stream);

/* Internal magnetisation state (checkpoint / resume), device N' x 3 T; set_m copies in,
 * get_m copies out.  set_m normalises nothing: pass unit vectors. */
int pmfem_set_m(pmfem_t h, const void* m, void* stream);
int pmfem_get_m(pmfem_t h, void* m, void* stream);

/*
 * nsteps classical RK4 steps of size dt [s] of Eq. 2 on the internal state, each with
 * four field evaluations and m <- m/|m| at the end of the step (norm taken in FP64).
 * The first call for a dt captures one step as a CUDA graph (on a private stream, after
 * synchronising stream) and every step replays it; per-launch timing (pmfem_profile) and
 * the surrogate run the launches directly.  dt <= 0 or nsteps < 0 -> EINVAL.
 */
int pmfem_llg_step(pmfem_t h, double dt, int nsteps, void* stream);

/*
 * Implicit midpoint steps of Eq. 2 with Newton-Krylov (the paper's way of integrating the
 * discrete LLG system, Sec. 2.2 and Sec. 4: implicit schemes whose Newton iterations solve
 * their linear systems with a preconditioned Krylov solver).  One step of size dt [s]:
 *   y = m_n + dt f((m_n + y)/2),  f(m) = -g [m x H(m) + alpha m x (m x H(m))],
 * g = gamma0 / (1 + alpha^2); the rule keeps |m| of every node (no renormalisation).  Newton
 * starts from y = m_n; each Newton iteration solves J d = -R by restarted GMRES, right-
 * preconditioned by 3x3 blocks per node (J with the field's linear part replaced by the
 * exchange operator's own coefficient), where every product J v costs one evaluation of the
 * field's linear part (the path of pmfem_field with PMFEM_EX | PMFEM_MS).  Works on the internal
 * state (pmfem_set_m / pmfem_get_m) at the handle's precision; synchronises stream at every
 * Krylov iteration (its scalars go to the host).
 *   opts   may be NULL; zero fields take the defaults:
 *            newton_tol  step converged when |d| <= newton_tol |y|   (1e-10 FP64, 1e-5 FP32)
 *            krylov_tol  GMRES relative residual per Newton step       (1e-8 FP64, 1e-4 FP32)
 *            restart     GMRES cycle length, 1..64                      (30)
 *            max_newton  Newton iterations per step                     (20)
 *            max_krylov  GMRES iterations per Newton iteration          (600)
 *   stats  host int64[4] or NULL: Newton iterations, Krylov iterations, field evaluations,
 *          steps completed (also on failure).
 * ENOCONV when Newton does not converge: the state stays at the start of the failed step.
 * EINVAL for dt <= 0, nsteps < 0, restart > 64 or a tolerance >= 1.
 */
typedef struct pmfem_implicit_opts {
  double newton_tol;
  double krylov_tol;
  int restart;
  int max_newton;
  int max_krylov;
} pmfem_implicit_opts;
int pmfem_llg_step_implicit(pmfem_t h, double dt, int nsteps, const pmfem_implicit_opts* opts, int64_t* stats,
                            void* stream);

/*
 * Bloch-phase periodic Green's function (Eq. 15 with k0 != 0; Sec. 4.3 excites phase-shifted
 * periodic sources): G_k(r) = sum_l e^{-j k0.l} / |r - l| over the lattice of the handle's
 * periodic axes, k0 (host, 3 doubles, rad/m) along those axes and off their reciprocal lattice.
 * With q~ = q e^{j k0.r} and the twisted kernel K~(d) = G_k(d) e^{j k0.d}, which is periodic
 * and Hermitian, the potential of quasi-periodic sources is e^{-j k0.r} times the circular
 * convolution of q~ with K~ on the grid of Eq. 16 (BAIM step 2; open axes zero-padded to 2N).
 *
 * pmfem_bloch_spectrum: the spectrum of K~ on the FFT grid, computed on the GPU in FP64 (Ewald
 * sums as for k0 = 0, plus its discrete transform): out host fft[0] x fft[1] x fft[2] doubles,
 * x fastest, unscaled; it is real (max_imag, host double or NULL, receives the largest
 * imaginary part of the transform).  Synchronises the device.
 * pmfem_bloch_convolve: U~ = the convolution of Q~ with K~ on the node grid, Q and U device
 * dims[0] x dims[1] x dims[2] complex numbers (interleaved re, im) of the precision's type T,
 * x fastest; enqueued on stream.  The spectrum of the last k0 is kept on the device.
 * The transforms are the radix-2 line transforms of BAIM step 2, complex to complex over the full
 * FFT grid (the twisted kernel's spectrum is real but not even): FP64 for the spectrum, the
 * precision's type T for the convolution, O(log F) work per point and axis.  The first call for
 * a k0 (or after a precision change) sets up that spectrum and synchronises the device; later
 * calls with the same k0 only enqueue the five passes.  EINVAL for k0 off the periodic axes or on
 * the reciprocal lattice, checked before any device work; ESTATE before pmfem_set_periodicity.
 */
int pmfem_bloch_spectrum(pmfem_t h, const double* k0, double* out, double* max_imag);
int pmfem_bloch_convolve(pmfem_t h, const double* k0, const void* Q, void* U, void* stream);

/*
 * Per-launch timing for measurement.  pmfem_profile(h, 1) starts recording a CUDA event
 * pair around every kernel the handle launches (on the stream it launches on) and clears
 * the totals; 0 stops recording.  pmfem_profile_read synchronises the device and writes,
 * for kernel ids 0..n-1, the launch counts and the summed event time in ms since the last
 * pmfem_profile(h, 1).  Ids: 0 charges, 1 projection, 2 FFT x forward, 3 FFT y forward,
 * 4 FFT z + spectral multiply, 5 FFT y inverse, 6 FFT x inverse, 7 interpolation +
 * precorrection (the precorrection alone where the two-pass form runs), 8 gradient + exchange
 * (+ RK4 stage), 9 grid clear, 10 permutation between the C-ABI unknown order and the internal
 * box-sorted order, 11 stencil of the grid potential added to the precorrected potential (the
 * second pass of the two-pass form, in which the precorrection runs on a second stream beside the
 * projection and the FFT; with timing on, every launch runs on the launching stream in order),
 * 12, 13, 14 the surrogate network's 1 -> 32, 32 -> 32 (both hidden layers) and 32 -> 1 layers
 * (pmfem_surrogate_apply and the surrogate's RK stages).
 */
int pmfem_profile(pmfem_t h, int enable);
int pmfem_profile_read(pmfem_t h, int64_t* counts, double* total_ms, int n);

/* Wait for all work of the handle; returns ENONFINITE / ETIMEOUT if a device check fired
 * since the previous sync (the flag is then cleared). */
int pmfem_sync(pmfem_t h);
int pmfem_destroy(pmfem_t h);

/*
 * Introspection of the host set-up (for tests and tools; host pointers, FP64).
 *   which: 0 exchange  K'_nk  = -(2A/(mu0 Ms)) K_nk / V_n                       (1 comp)
 *          1 charges   W'_nk  = Ms (W^q)_nk                                      (3 comp)
 *          2 near-element E'_nk = Ms E_nk on the adjacency pattern               (3 comp)
 *          3 gradient  G'_nk  = -(W^q)_kn / (4 pi V_n)                           (3 comp)
 *          4 point precorrection C_nk                                             (1 comp)
 *          5 near-element entries outside the adjacency pattern                   (3 comp)
 *   info gives rows, nnz and components; export fills rowptr (rows+1), col (nnz) and
 *   vals (nnz x comp, row-major).
 */
int pmfem_operator_info(pmfem_t h, int which, int64_t* rows, int64_t* nnz, int* comps);
int pmfem_operator_export(pmfem_t h, int which, int32_t* rowptr, int32_t* col, double* vals);

/*
 * Device layout facts (uploads the device data for the current precision if needed):
 * out[0..2] adjacency entries, padded SELL slots, column bits; out[3..5] the same for the
 * point precorrection; out[6..8] for the projection; out[9] projection exception entries;
 * out[10..11] box-order tile rows and planes; out[12] rows of the projection (the grid points
 * that some node projects to; the grid is cleared before each projection).
 */
int pmfem_device_info(pmfem_t h, int64_t* out, int n);

/*
 * Test and diagnosis hooks (no counterpart in the paper).
 * pmfem_debug_fail_alloc: process-wide; after `after` more device allocations of the library
 * succeed, every further one fails with ENOMEM without calling the CUDA allocator, so that the
 * out-of-memory paths (and the clean-up of a partial device build) can be tested without
 * exhausting a GPU.  -1 switches it off (the default); EINVAL below -1.
 * pmfem_build_flags: bit 0 set in a PMFEM_CHECKS build, which checks every stored index of a
 * device upload against its bounds on the device (a failure is reported by pmfem_sync as
 * EINVAL) and clamps gathered indices into their vectors.
 */
int pmfem_debug_fail_alloc(int after);
int pmfem_build_flags(void);

/*
 * Wall-clock seconds of the set-up stages of the handle (host, n doubles; stages beyond 7
 * read 0): out[0] PBC pairing and fold (Sec. 2.2, Eq. 18), out[1] periodized local operators
 * (Eqs. 7-12, 14a, 14d), out[2] grid and stencils (Eq. 16), out[3] PGF spectrum (Eq. 15),
 * out[4] near-element correction (Eq. 14c), out[5] point precorrection (BAIM step 4), all of
 * the last pmfem_set_periodicity; out[6] device layout and upload of the last device build.
 */
int pmfem_setup_times(pmfem_t h, double* out, int n);

/* Grid of Eq. 16 as set up: dims[3], fft[3], origin[3], delta[3] (host). */
int pmfem_grid_info(pmfem_t h, int32_t* dims, int32_t* fft, double* origin, double* delta);
/* PGF spectrum (Eq. 15 on the grid, transformed), reduced by symmetry:
 * (fft[0]/2+1) x (fft[1]/2+1) x (fft[2]/2+1) doubles, x fastest, unscaled. */
int pmfem_export_spectrum(pmfem_t h, double* out);
/* Folded unknown positions of Eq. 18 (host, N' x 3 doubles). */
int pmfem_folded_positions(pmfem_t h, double* out);

/* ======================================================================================
 * Learned surrogate of the FFT convolution (the paper has no counterpart).  A 3D
 * convolutional network on the handle's AIM grid (Eq. 16) maps grid charges Q (BAIM step 1)
 * to grid potential U (what step 2, the FFT convolution with the PGF of Eq. 15, gives):
 *   h1 = act(conv(Q / sq)), h2 = act(conv(h1)), h3 = act(conv(h2)), U = su * conv(h3),
 * 3x3x3 kernels, 1 -> 32 -> 32 -> 32 -> 1 channels with biases, act(z) = z (z > 0) or
 * 0.1 z, circular padding along periodic axes and zero padding along the others.  Grids are
 * device arrays of N0 x N1 x N2 FP32 (x fastest; pmfem_grid_info gives the dimensions, which
 * must be multiples of 8, 8 and 4).  Weights, gradients and accumulation are FP32; hidden
 * activations are FP32 or, with act_bf16, bfloat16.  With bfloat16 activations on a grid
 * whose x and y dimensions are multiples of 8 and 16, the two 32 -> 32 layers run on the
 * tensor cores (tcgen05, BF16 operands, FP32 accumulation).  Training minimises the mean squared
 * error (in units of su) with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * ====================================================================================== */

/*
 * Create (or reset) the handle's network with the given parameters: host, n = 57121 floats,
 * layer after layer W[co][ci][dz][dy][dx] then b[co]; sq, su > 0.  Resets the Adam state.
 * ESTATE before pmfem_set_periodicity; EINVAL for a wrong count, a non-finite value or a
 * grid that is not a multiple of (8, 8, 4).
 */
int pmfem_surrogate_set_params(pmfem_t h, const float* params, int64_t n, double sq, double su, int act_bf16);
int pmfem_surrogate_get_params(pmfem_t h, float* params);                     /* host, 57121 floats */
/* U = net(Q) for one grid (device arrays). */
int pmfem_surrogate_apply(pmfem_t h, const float* Q, float* U, void* stream);
/* Gradient (host, 57121 floats, parameter order) and loss of one pair; synchronous. */
int pmfem_surrogate_grad(pmfem_t h, const float* Q, const float* U, float* grads, double* loss);
/*
 * Train on npairs pairs (device, npairs x grid each), in order, for epochs passes; an Adam
 * step after every batch pairs, with learning rate lr.  epoch_loss (host, epochs doubles,
 * may be NULL) receives the mean loss of every pass.
 */
int pmfem_surrogate_train(pmfem_t h, const float* Q, const float* U, int64_t npairs, int epochs, int batch, double lr,
                          double* epoch_loss, void* stream);
/* Training data from the method itself: for a magnetisation m (device N' x 3 FP32), the grid
 * charges Q of step 1 and the FFT potential U of step 2 (FP32 path; ESTATE under FP64). */
int pmfem_grid_pair(pmfem_t h, const void* m, float* Q, float* U, void* stream);
/*
 * every_k > 0: pmfem_llg_step (FP32) runs the full P-AIM on the first RK stage of every step
 * and keeps its Q1 and U1; stages 2-4 use U = U1 + net(Q - Q1) in place of the FFT, except
 * on every every_k-th step (the first included), where they run the full P-AIM and the
 * network's potential is measured against it.  0 switches it off.  Resets the statistics.
 */
int pmfem_surrogate_enable(pmfem_t h, int every_k);
/* out[4]: steps taken, stages that used the network, stages judged, and the relative L2
 * error of the network's potential over all judged stages (sqrt(sum |dU|^2 / sum |U|^2)).
 * Synchronises; ETIMEOUT if a tensor-core convolution gave up waiting for its MMAs. */
int pmfem_surrogate_stats(pmfem_t h, double* out);

/* ======================================================================================
 * Batches of independent cells (the paper has no counterpart: a service for sweeps such as
 * a hysteresis loop, where many unit cells, each with its own applied field, advance
 * together).  A batch evaluates the field of every cell and advances every cell by RK4 in
 * FP32, as pmfem_field / pmfem_llg_step would for each cell alone, but each pass runs as one
 * launch over the rows of all cells (one FFT launch per group of cells with the same grid
 * shape), and a whole RK4 step is replayed from a captured CUDA graph.
 *
 * Arrays of a batch are device N_tot x 3 FP32, the cells' unknowns concatenated in cell
 * order (pmfem_batch_offsets gives where each cell starts).
 * ====================================================================================== */
typedef struct pmfem_batch_state* pmfem_batch_t;

/*
 * Batch of n cells (n >= 1).  Every cell must be set up (pmfem_set_periodicity done, else
 * ESTATE) and all must use the same stencil order p (else EINVAL).  The batch keeps the
 * handles, which must outlive it; it reads each cell's set-up, layout settings and applied
 * field when it builds its device data (at the first call that needs them).  The cells
 * stay usable on their own.  *out is NULL on failure.
 */
int pmfem_batch_create(pmfem_batch_t* out, const pmfem_t* cells, int n);
int pmfem_batch_destroy(pmfem_batch_t b);
const char* pmfem_batch_last_error(pmfem_batch_t b);

/* offsets (host, n + 1): cell c owns unknowns [offsets[c], offsets[c + 1]). */
int pmfem_batch_offsets(pmfem_batch_t b, int64_t* offsets);

/*
 * Box-order tiles by measurement (autotuner): for every cell, each candidate tile shape
 * (tile rows x tile planes: 8x4, 8x2, 4x4, 16x2, 4x2) is set with pmfem_set_layout, the
 * cell's own FP32 field is timed (reps evaluations, CUDA events, after one warm-up), and the
 * fastest is kept.  Results are cached for the process per (grid shape, FFT shape, N'
 * within a factor 2^(1/4)), so cells alike are tuned once.  Changes the cells' layout
 * settings, drops the batch's device data (the state m included; the next call rebuilds
 * it) and synchronises.  reps in [1, 100], else EINVAL.
 */
int pmfem_batch_autotune(pmfem_batch_t b, int reps);
/* tiles (host, 2n): the (tile rows, tile planes) of every cell's box order in the batch's
 * device data (builds it if needed). */
int pmfem_batch_tiles(pmfem_batch_t b, int32_t* tiles);

/* Applied field of cell c (A/m, uniform), enqueued on stream: later evaluations and graph
 * replays use it.  EINVAL for c outside [0, n). */
int pmfem_batch_set_applied_field(pmfem_batch_t b, int c, double Hx, double Hy, double Hz, void* stream);

/* Field of every cell (as pmfem_field, FP32): m and H device N_tot x 3 FP32. */
int pmfem_batch_field(pmfem_batch_t b, const void* m, void* H, int components, void* stream);

/* State of every cell (device N_tot x 3 FP32); set_m normalises nothing. */
int pmfem_batch_set_m(pmfem_batch_t b, const void* m, void* stream);
int pmfem_batch_get_m(pmfem_batch_t b, void* m, void* stream);

/*
 * nsteps RK4 steps of size dt (> 0, seconds) of every cell, as pmfem_llg_step.  The first
 * call for a given dt captures one step into a CUDA graph (on a stream of the library) and
 * every step replays it on stream.  A cell's applied field is read by the graph at every
 * replay.  EINVAL for dt <= 0 or nsteps < 0.
 */
int pmfem_batch_llg_step(pmfem_batch_t b, double dt, int nsteps, void* stream);

/* Waits for the device and reports a device error of the batch (ENONFINITE) like pmfem_sync. */
int pmfem_batch_sync(pmfem_batch_t b);

/*
 * Per-launch timing of the batch's kernels, as pmfem_profile / pmfem_profile_read with the same
 * kernel ids (the batch runs the fused interpolation + precorrection, id 7, and no stencil
 * pass).  While timing is on, pmfem_batch_llg_step launches every kernel in order on its stream
 * instead of replaying its captured step, so that each launch is timed alone.
 */
int pmfem_batch_profile(pmfem_batch_t b, int enable);
int pmfem_batch_profile_read(pmfem_batch_t b, int64_t* counts, double* total_ms, int n);

#ifdef __cplusplus
}
#endif
#endif /* PMFEM_H */
