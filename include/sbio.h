/*
 * sbio.h -- C ABI of the GB300 spheroidal boundary-integral-operator library.
 *
 * The library applies the Laplace single-layer (S) and double-layer (D)
 * operators, and the Stokes single layer through the Laplace-to-Stokes
 * identity, to densities given as spheroidal-harmonic coefficients on a
 * suspension of prolate and oblate spheroids, at every surface quadrature node
 * ("Boundary integral equation analysis for spheroidal suspensions", Sec. 4,
 * eq. (potall) and Algorithm 1; Stokes: Sec. 4.3, eq. (stokes)).
 *
 * Conventions shared by every entry point
 *   - Return value: SBIO_OK (0) or a negative SBIO_E* code.  The message of the
 *     last failure on the calling thread is available from sbio_last_error().
 *   - Device pointers are plain CUDA device addresses of the context's device;
 *     host pointers are ordinary process memory.  The caller owns every buffer
 *     it passes; the library owns everything behind the opaque handles.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Apply calls are stream-ordered and asynchronous unless their
 *     description says otherwise; buffers must stay valid until the stream
 *     reaches the call.
 *   - Node order: particle-major, then Gauss-Legendre node j in v (ascending),
 *     then trapezoid node k in phi (phi_k = 2 pi k / n_phi).  A suspension of M
 *     particles at order p has N = M (p+1) n_phi targets.
 *   - Coefficient order: per particle, index n*n + n + m for 0 <= n <= p,
 *     -n <= m <= n, in the real orthonormal surface-harmonic basis
 *     (m > 0: sqrt(2) N_n^m P_n^m(v) cos(m phi); m = 0: N_n^0 P_n(v);
 *     m < 0: sqrt(2) N_n^|m| P_n^|m|(v) sin(|m| phi)), Definition 1 with
 *     Ferrers functions without the Condon-Shortley phase.
 *   - Geometry and outputs are FP64 in every precision mode.
 *   - A geometry handle may be used by one thread at a time; calls that
 *     overlap on the GPU through the same geometry share its workspaces and
 *     race, so issue them on one stream.
 */
#ifndef SBIO_H
#define SBIO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define SBIO_OK 0
#define SBIO_EINVAL (-1)    /* bad argument: sizes, p, shape, quaternion, pointer */
#define SBIO_EOVERLAP (-2)  /* a surface node lies inside another spheroid */
#define SBIO_ENOMEM (-3)    /* allocation failed or the context budget is exceeded */
#define SBIO_ECUDA (-4)     /* a CUDA runtime call failed */
#define SBIO_ETIMEOUT (-5)  /* a bounded device-side wait expired */
#define SBIO_ENOTSUP (-6)   /* valid request this build does not implement */

/* ---- particle kinds, precision modes, parts -------------------------- */
#define SBIO_PROLATE 0
#define SBIO_OBLATE 1

#define SBIO_FP64 0   /* every kernel in FP64 */
#define SBIO_MIXED 1  /* far-field pair sums in FP32 with two-sum compensated
                         accumulation; self term in FP64; the S + D near
                         field with coordinates, Q recurrences and angles in
                         FP64 and the Ferrers recurrence and the
                         contraction in compensated FP32 (the derivative,
                         Stokes and double-layer near fields stay FP64) */

#define SBIO_PART_SELF 1u  /* on-surface self interaction (Sec. 4.1 "Near-field") */
#define SBIO_PART_NEAR 2u  /* neighbour particles by the exterior expansion */
#define SBIO_PART_FAR 4u   /* smooth quadrature over far particles (Sec. 4.1) */
#define SBIO_PART_ALL 7u

#define SBIO_MAX_P 24      /* largest expansion order accepted */

typedef struct sbio_ctx sbio_ctx;   /* opaque: device, memory budget, error state */
typedef struct sbio_geom sbio_geom; /* opaque: resident geometry of one suspension */

/* One spheroid (Sec. 2.1, Table 1; Sec. 5.1 problem statement).
 *   kind: SBIO_PROLATE (C > A) or SBIO_OBLATE (C < A); spheres are rejected.
 *   A: equatorial semi-axis, C: polar semi-axis along the local x3 axis.
 *   center: global position; quat: unit quaternion (w, x, y, z) with
 *   x_global = center + R(quat) x_local.  Quaternions are normalised if their
 *   norm is within 1e-6 of 1, otherwise SBIO_EINVAL. */
typedef struct {
  int32_t kind;
  int32_t reserved;
  double A;
  double C;
  double center[3];
  double quat[4];
} sbio_spheroid;

/* Discretisation and method options.
 *   p: expansion order, 1 <= p <= SBIO_MAX_P (Sec. 4, (p+1)^2 coefficients).
 *   n_phi: trapezoid nodes in phi; 0 selects 2(p+1) (the paper prints 2p;
 *          with 2p the sin(p phi) mode vanishes at every node).
 *   near_factor: target x is near to particle i iff the exact distance from x
 *          to the surface of i is below near_factor * (major semi-axis of i)
 *          (Sec. 4.1 with eta = near_factor / 2); must be > 0.
 *   far_upsample: must be 1 (far sources are the same quadrature nodes).
 *   precision: SBIO_FP64 or SBIO_MIXED. */
typedef struct {
  int32_t p;
  int32_t n_phi;
  double near_factor;
  int32_t far_upsample;
  int32_t precision;
} sbio_options;

/* Library version string (static storage). */
const char* sbio_version(void);

/* Message of the last failure on the calling thread ("" if none).  `ctx` may
 * be NULL.  The pointer stays valid until the next failing call on the thread. */
const char* sbio_last_error(const sbio_ctx* ctx);

/* Number of kernels this process has launched through the library so far
 * (all contexts); used to count launches inside a timed region. */
int64_t sbio_launch_count(void);

/* Measured pipe rates of one GPU (no counterpart in the paper: the roofline
 * denominators of the hot path's kernels, which no copy or GEMM benchmark
 * gives).  Each rate comes from a kernel of independent dependency chains at
 * full occupancy (8 CTAs of 256 threads per SM), timed with CUDA events after
 * a warm-up launch on a private stream:
 *   fp32_ffma_tflops / fp32_ffma2_tflops: scalar FMA and packed f32x2 FMA
 *     (2 flop per FMA);
 *   rsqrt_per_s: MUFU rsqrt.approx.f32 per second;
 *   fp64_dfma_tflops: FP64 FMA;
 *   pairmix_pairs_per_s: far-field S + D pairs per second with the packed
 *     far kernel's register arithmetic per two pairs (11 f32x2 instructions,
 *     2 rsqrt) and no memory traffic, i.e. the rate the far kernel could
 *     reach if staging and bookkeeping cost nothing;
 *   pairsmem_pairs_per_s: the same pairs with the sources read from shared
 *     memory as the far kernel reads them (five 16-byte loads per source,
 *     8 targets per thread) but without tiles, skip lists or barriers;
 *   sm_clock_mhz: SM clock during the kernels (%clock64 over %globaltimer);
 *   sms: multiprocessor count.
 * Synchronous; allocates 48 bytes of device memory for the duration of the
 * call.  Errors: SBIO_EINVAL (device out of range, null out), SBIO_ECUDA. */
typedef struct {
  double fp32_ffma_tflops;
  double fp32_ffma2_tflops;
  double rsqrt_per_s;
  double fp64_dfma_tflops;
  double pairmix_pairs_per_s;
  double pairsmem_pairs_per_s;
  double sm_clock_mhz;
  int32_t sms;
  int32_t reserved;
} sbio_peaks;
int sbio_measure_peaks(int32_t device, sbio_peaks* out);

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the
 * device memory that geometries of this context may hold (0 = no bound);
 * geometry creation that would exceed it fails with SBIO_ENOMEM. */
int sbio_ctx_create(int device, size_t mem_budget_bytes, sbio_ctx** out);

/* Destroy a context.  All its geometries must have been destroyed. */
int sbio_ctx_destroy(sbio_ctx* ctx);

/* Device bytes currently held by geometries of the context. */
int sbio_ctx_mem_used(const sbio_ctx* ctx, size_t* bytes);

/* Build the resident geometry of a suspension (host FP64 set-up, then upload
 * on `stream`; the call returns after the upload has completed):
 *   spheroid parameters a, u0 from the semi-axes (Sec. 2.1), rotations,
 *   quadrature nodes, outward normals and weights w = w_j^GL (2 pi / n_phi)
 *   dS-factor (Table 2), the per-particle multipliers of Theorems 1-2 and the
 *   per-target near sets (Sec. 4.1).
 *   sph: host array of M descriptors; M >= 1.
 * Errors: SBIO_EINVAL (bad options or shapes), SBIO_EOVERLAP (a node of one
 * particle lies inside another), SBIO_ENOMEM, SBIO_ECUDA. */
int sbio_geom_create(sbio_ctx* ctx, const sbio_spheroid* sph, int32_t M,
                     const sbio_options* opts, void* stream, sbio_geom** out);

/* Release a geometry (synchronises the device first). */
int sbio_geom_destroy(sbio_geom* g);

/* Sizes of a geometry: targets N, (target, near particle) pairs, (target,
 * far source node) pairs of one apply, and the device bytes it holds.  Any
 * output pointer may be NULL. */
int sbio_geom_info(const sbio_geom* g, int64_t* n_targets, int64_t* n_near_pairs,
                   int64_t* n_far_pairs, size_t* device_bytes);

/* Wall-clock milliseconds of the geometry's creation: host nodes and
 * multipliers, host near sets, device tables and upload (any may be NULL). */
int sbio_geom_setup_times(const sbio_geom* g, double* host_ms, double* near_ms, double* device_ms);

/* Copy node data to host arrays (any may be NULL): global positions (N x 3),
 * outward unit normals (N x 3), quadrature weights (N). */
int sbio_geom_nodes(const sbio_geom* g, double* xyz, double* normal, double* weight);

/* Copy the near pairs to host arrays of length n_near_pairs: target node index
 * and source particle index, in the library's processing order. */
int sbio_geom_near_pairs(const sbio_geom* g, int32_t* target, int32_t* source);

/* Phase timing (measurement aid).  When enabled, every Laplace apply records
 * CUDA events on its stream before the synthesis kernel, before the near-field
 * kernels, before the far-field kernel and after it (the Stokes applies and
 * S' / D' likewise, their prep and self kernels counting as the first phase),
 * with the phases run in order.  sbio_geom_phase_times()
 * synchronises on those events and returns the three durations of the last
 * apply in milliseconds (SBIO_EINVAL if timing is off). */
int sbio_geom_enable_timing(sbio_geom* g, int32_t on);

/* Work of the S + D near field (Algorithm 1, near branch), for the roofline
 * count: n_pairs (target, near particle) pairs, and miller_steps = the sum
 * over the pairs of the rolled backward-recurrence steps the kernel runs
 * above the top order before its unrolled part (about 19 / acosh(u) or
 * 19 / asinh(u) per pair, data dependent).  Runs one counting kernel on the
 * legacy default stream and synchronises.  Either output may be NULL. */
int sbio_geom_near_work(sbio_geom* g, int64_t* n_pairs, int64_t* miller_steps);
int sbio_geom_phase_times(sbio_geom* g, double* ms_synth, double* ms_near, double* ms_far);

/* Launch shape of the far-field kernels: far_tt targets per thread of the
 * mixed kernel (1, 2, 4 or 8; -2, -4, -8 select the same counts computed two
 * targets per packed f32x2 instruction) and far_splits source splits of the grid (0 =
 * chosen from the device's SM count).  Results do not depend on the shape
 * beyond floating-point summation order. */
int sbio_geom_set_launch_shape(sbio_geom* g, int32_t far_tt, int32_t far_splits);

/* Near-field CTAs per SM while the near field overlaps the far field (grid-
 * stride near kernels; 0 = one CTA per 128 pairs, no cap).  Default 2. */
int sbio_geom_set_near_cap(sbio_geom* g, int32_t ctas_per_sm);

/* Current launch shape (outputs may be NULL). */
int sbio_geom_get_tuning(const sbio_geom* g, int32_t* far_tt, int32_t* far_splits, int32_t* near_ctas_per_sm);

/* Autotuner: times the far-field kernel of this geometry in its current
 * precision mode for a small set of launch shapes (CUDA events on `stream`,
 * zero-strength sources written by one self-only pass into the geometry's
 * own workspaces) and keeps the fastest; then, when the near field overlaps
 * the far field, times whole applies for a few near CTA caps and keeps the
 * fastest (with a treecode attached, also the treecode's own near cap, by
 * whole applies with the treecode).  The direct kernel's shape is tuned with
 * the direct sum also when a treecode is attached.  Reports the far shape
 * (outputs may be NULL).  Synchronises `stream`; the workspaces hold no
 * caller data afterwards. */
int sbio_geom_autotune(sbio_geom* g, void* stream, int32_t* far_tt, int32_t* far_splits, double* far_ms);

/* Near/far overlap (default on): the near-field kernels of an apply run
 * on a high-priority stream forked from the caller's stream, beside the FP32
 * far-field kernel, and are joined back before the call's work ends on the
 * caller's stream.  Phase timing (sbio_geom_enable_timing) runs the phases in
 * order instead.  Off: everything on the caller's stream. */
int sbio_geom_set_overlap(sbio_geom* g, int32_t on);

/* Change the precision mode used by later applies (SBIO_FP64 / SBIO_MIXED). */
int sbio_geom_set_precision(sbio_geom* g, int32_t precision);

/* Laplace apply at all N surface nodes (Algorithm 1 for D; its single-layer
 * variant for S, Sec. 4.2):
 *   S_out[t] = S[sigma](x_t),  sigma = sum sigma~_nm Y_nm / sqrt(u0^2 -+ v^2)
 *              (modified basis, Sec. 3.2);
 *   D_out[t] = D[mu](x_t),     mu = sum mu^_nm Y_nm, principal value on the
 *              own surface (Theorem 1).
 * sigma_tilde, mu_hat: device, M x (p+1)^2 FP64, or NULL to skip that operator.
 * S_out, D_out: device, N FP64, must be non-NULL iff the matching input is.
 * Outputs are overwritten.  Asynchronous on `stream`. */
int sbio_apply_laplace(sbio_geom* g, const double* sigma_tilde, const double* mu_hat,
                       double* S_out, double* D_out, void* stream);

/* As sbio_apply_laplace, restricted to a subset of the three parts
 * (SBIO_PART_* bit mask); the outputs hold the sum of the selected parts. */
int sbio_apply_laplace_parts(sbio_geom* g, const double* sigma_tilde, const double* mu_hat,
                             double* S_out, double* D_out, uint32_t parts, void* stream);

/* One-sided surface limits (Sec. 2.4, jump conditions): as sbio_apply_laplace
 * with, on every node's own surface, side = +1 the exterior limit
 * D+ = D + mu/2 or side = -1 the interior limit D- = D - mu/2 (mu the
 * density value at the node; side = 0 the principal value, as
 * sbio_apply_laplace).  S is continuous and is the same for every side.
 * SBIO_EINVAL for side outside {-1, 0, 1}.  Asynchronous. */
int sbio_apply_laplace_limit(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* S_out,
                             double* D_out, int32_t side, void* stream);

/* End-to-end apply from and to HOST memory: copies the coefficients to
 * library-owned device buffers on `stream`, applies, copies the results back
 * and synchronises `stream` before returning.  Host buffers may be pageable or
 * pinned (pinned gives overlap-free fast copies). */
int sbio_apply_laplace_host(sbio_geom* g, const double* sigma_tilde_host, const double* mu_hat_host,
                            double* S_host, double* D_host, void* stream);

/* Stokes single layer with viscosity 1 at all N nodes (Sec. 4.3, eq. (stokes)):
 *   u_k = 1/2 { S[f_k] - sum_j x_j d_k S[f_j] + d_k S[y . f] },  k = 1..3,
 * far particles by the Stokeslet quadrature, near and self by the Laplace
 * expansions and their gradients (eq. (dSLevalformula)).
 * f_tilde: device, M x 3 x (p+1)^2 FP64: per particle the modified-basis
 *          coefficients of the three global Cartesian components of f.
 * u_out: device, N x 3 FP64 (row t = velocity at node t).  Asynchronous. */
int sbio_apply_stokes_sl(sbio_geom* g, const double* f_tilde, double* u_out, void* stream);

/* Normal derivatives of the layer potentials at all N nodes (Sec. 3.3,
 * Theorem 3 and eq. (dSLevalformula); Sec. 4.2 "Other layer potentials"):
 *   Sp_out[t] = S'[sigma](x_t) = d/dnu(x_t) S[sigma](x_t), on the own surface
 *               the principal value (average of the exterior and interior
 *               limits; S'+ = S' - sigma/2, S'- = S' + sigma/2),
 *   Dp_out[t] = D'[mu](x_t) = d/dnu(x_t) D[mu](x_t) (continuous across the
 *               surface; hypersingular, evaluated through the multipliers),
 * nu the outward unit normal at the target node.  Inputs, layouts, precision
 * modes, near sets and the far-field rule are those of sbio_apply_laplace
 * (either input may be NULL; each output is given exactly when its input
 * is); outputs overwritten.  SBIO_ENOTSUP for p > 20.  Asynchronous. */
int sbio_apply_laplace_deriv(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* Sp_out,
                             double* Dp_out, void* stream);

/* One-sided limits of the normal derivatives: as sbio_apply_laplace_deriv
 * with side = +1 the exterior limit S'+ = S' - sigma/2 or side = -1 the
 * interior limit S'- = S' + sigma/2 on every node's own surface (sigma the
 * density value at the node; side = 0 the principal value).  D' is
 * continuous and is the same for every side.  SBIO_EINVAL for side outside
 * {-1, 0, 1}.  Asynchronous. */
int sbio_apply_laplace_deriv_limit(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* Sp_out,
                                   double* Dp_out, int32_t side, void* stream);

/* Stokes double layer (viscosity 1) at all N nodes, principal value:
 *   D_stk[q](x)_i = 3/(4 pi) int (r.q)(r.nu) r_i / |r|^5 dS, r = x - y,
 * nu the outward normal (the sign that makes D_stk[const] = -q inside and
 * -q/2 on the surface, like sbio_apply_laplace's D).  The paper only remarks
 * (Sec. 4.3) that the Stokes double layer can be evaluated through Laplace
 * potentials; here D_stk_i = -x_i sum_j d_j D[q_j] + sum_j d_j D[y_i q_j] -
 * d_i S[q.nu] for near and own pairs (thirteen expansions, exact at order
 * p+1) and the stresslet quadrature for far pairs.  q_hat: device,
 * M x 3 x (p+1)^2 plain coefficients (the D input convention) of the three
 * Cartesian components; u_out: device, N x 3, overwritten.  SBIO_ENOTSUP for
 * p > 20.  Asynchronous. */
int sbio_apply_stokes_dl(sbio_geom* g, const double* q_hat, double* u_out, void* stream);

/* One-sided limits of the Stokes double layer on every node's own surface:
 * side = +1 the exterior limit (principal value + q/2), side = -1 the
 * interior limit (principal value - q/2), side = 0 the principal value (as
 * sbio_apply_stokes_dl); q the density at the node.  SBIO_EINVAL for side
 * outside {-1, 0, 1}.  Asynchronous. */
int sbio_apply_stokes_dl_limit(sbio_geom* g, const double* q_hat, double* u_out, int32_t side, void* stream);

/* End-to-end Stokes apply from and to HOST memory (f_tilde_host M x 3 x
 * (p+1)^2, u_host N x 3): copies in through library-owned device buffers on
 * `stream`, applies, copies out and synchronises `stream` before returning. */
int sbio_apply_stokes_sl_host(sbio_geom* g, const double* f_tilde_host, double* u_host, void* stream);

/* Launch settings of the Stokes kernels, kept apart from the Laplace ones
 * (the Stokeslet far kernel carries three accumulators per target and its
 * near field is the larger share of an apply): far_tt and far_splits as in
 * sbio_geom_set_launch_shape, near_ctas_per_sm as in sbio_geom_set_near_cap
 * (default 2, 0, 0).  The double layer's stresslet far kernel follows a
 * packed far_tt (-2, -4, -8, with far_splits) and otherwise runs its scalar
 * form with 4 targets per thread.  SBIO_EINVAL on values outside those sets. */
int sbio_geom_set_stokes_tuning(sbio_geom* g, int32_t far_tt, int32_t far_splits, int32_t near_ctas_per_sm);
int sbio_geom_get_stokes_tuning(const sbio_geom* g, int32_t* far_tt, int32_t* far_splits, int32_t* near_ctas_per_sm);

/* Autotuner of the Stokes kernels: as sbio_geom_autotune, timing the
 * Stokeslet far kernel and whole Stokes applies (zero forces through the
 * geometry's own workspaces), near caps from 4 CTAs per SM up or uncapped
 * (the Stokes near kernels run small CTAs).  The velocity-and-pressure evaluation at
 * points runs its near pairs at twice the tuned near cap (its near pairs cost
 * about twice the single layer's).  SBIO_ENOTSUP for p > 20.  Synchronises
 * `stream`. */
int sbio_geom_autotune_stokes(sbio_geom* g, void* stream, int32_t* far_tt, int32_t* far_splits, double* far_ms);


/* ---- far field by a particle treecode -----------------------------------
 * The paper evaluates the far field with an FMM (Sec. 4.1 "Far-field"); past
 * a few hundred particles the O(N^2) direct sum here grows too slow, and a
 * treecode can replace it for mixed-precision applies at the nodes of the
 * Laplace S + D (sbio_apply_laplace / _parts / _host with both operators) and
 * of the Stokes single layer (sbio_apply_stokes_sl, its Stokeslet written as
 * 8 pi u_i = S[F_i] + (x - c)_i D[F] - D[(y - c)_i F] with F = w f, i.e.
 * four charge and four dipole channels about each node's centre c): a binary
 * tree
 * over the particles, solid-harmonic multipoles of order `order` (8, 12 or
 * 16) of every node's sources (charges q = w sigma for S, dipoles
 * d = w mu nu for D), accepted for a group of 256 consecutive targets when
 * every target is at least r_node / theta from the node's centre and the
 * node holds none of the group's own or near particles; every other particle
 * is summed directly with the per-target skip lists.  The result is the same
 * discrete far sum (Sec. 4.1 quadrature over the far particles' nodes) up to
 * the truncation of the expansions, about (theta)^(order+1) relative per
 * node (nodes farther than r_node / theta are evaluated at a lower order
 * with the same bound: sbio_geom_tree_order_counts).  SBIO_FAR_TREE builds the tree and lists on the host (synchronises
 * the device); SBIO_FAR_DIRECT (theta, order ignored) returns to the direct
 * sum.  FP64 geometries, evaluations at points and the other operators keep
 * the direct sum.  When the geometry overlaps its near field with the far
 * field (sbio_geom_set_overlap), an apply with the treecode runs the direct
 * part on a stream of the tree's own beside the multipole phases, and
 * SBIO_FAR_TREE also picks the near kernels' CTA cap for such applies by
 * timing whole Laplace applies of zero densities (kept apart from the direct
 * sum's cap: see sbio_geom_set_tree_near_cap; sbio_geom_autotune retunes it).
 * Errors: SBIO_EINVAL (method, theta outside (0.05, 1), order), SBIO_ENOMEM,
 * SBIO_ECUDA. */
#define SBIO_FAR_DIRECT 0
#define SBIO_FAR_TREE 1
int sbio_geom_set_far_method(sbio_geom* g, int32_t method, double theta, int32_t order);

/* Near-field CTAs per SM while the near field overlaps a treecode far field
 * (as sbio_geom_set_near_cap for the direct sum; default 2, 0 = no cap).
 * The getter's output may not be NULL.  SBIO_EINVAL for a negative cap. */
int sbio_geom_set_tree_near_cap(sbio_geom* g, int32_t ctas_per_sm);
int sbio_geom_get_tree_near_cap(const sbio_geom* g, int32_t* ctas_per_sm);

/* Sizes of the treecode far field per apply: tree nodes, target groups,
 * (target, multipole node) evaluations, the (target, source node) pairs those
 * evaluations stand for, and the (target, source node) pairs summed
 * directly; the last two add up to the geometry's far pair count (every far
 * pair is covered once).  SBIO_EINVAL if the geometry uses the direct sum. */
int sbio_geom_tree_info(const sbio_geom* g, int64_t* n_nodes, int64_t* n_groups, int64_t* m2p_pairs,
                        int64_t* m2p_source_pairs, int64_t* direct_pairs);

/* The (target, multipole node) evaluations per apply of operator `op`
 * (SBIO_OP_LAPLACE: S + D; SBIO_OP_STOKES: the Stokes single layer) by
 * evaluation order: evals[0], [1], [2] at orders 8, 12 and 16 (they add up
 * to m2p_pairs of sbio_geom_tree_info).  An accepted node is evaluated at the
 * lowest of these orders E (at most the treecode's order P) with
 * rho^(E+1) <= s theta^(P+1), rho = r_node / (distance from the target
 * group's centre to the node's centre - the group's radius) <= theta, and
 * s = 1 for Laplace (the truncation bound of every evaluation stays that of
 * order P at theta), s = 1/10 for Stokes (eight channels per node).
 * SBIO_EINVAL for a null argument, an unknown operator or a geometry
 * without a treecode. */
int sbio_geom_tree_order_counts(const sbio_geom* g, int32_t op, int64_t* evals);

/* Durations (ms) of the treecode phases of the last apply made with phase
 * timing on (sbio_geom_enable_timing): ms[0] leaf multipoles, ms[1]
 * translations up the tree and the FP32 copy, ms[2] the direct part, ms[3]
 * the multipole evaluations.  Synchronises on the last phase's event.
 * SBIO_EINVAL if the far field is direct or timing is off. */
int sbio_geom_tree_phase_times(sbio_geom* g, double* ms);

/* ---- particle-to-target evaluation (Sec. 4.1, "Particle-to-target
 * algorithm") ---------------------------------------------------------------
 * S[sigma] and D[mu] of every spheroid of a geometry at T arbitrary points in
 * the fluid (outside every spheroid).  The classification is per point: the
 * pair (point, spheroid i) is near iff the exact distance from the point to
 * the surface of i is below near_factor x (major semi-axis of i), the same
 * rule as for surface nodes; near pairs use the exterior expansions of
 * Theorems 1-2, all other pairs the smooth GL x trapezoid quadrature.
 * A target set is resident like the geometry it belongs to: creation
 * classifies the points on the host and uploads the pair lists; every
 * evaluation then runs on the device only. */
typedef struct sbio_targets sbio_targets;   /* opaque: points, near pairs, skip lists */

/* xyz_host: T x 3 global coordinates (host, row-major), copied.  Points on a
 * surface to rounding (level-set value within 1e-11 of 1) count as exterior
 * points; a point inside a spheroid fails with SBIO_EINVAL.  T = 0 is
 * allowed.  The set must be destroyed before its geometry (sbio_geom_destroy
 * returns SBIO_EINVAL while sets are alive).  Synchronises `stream`. */
int sbio_targets_create(sbio_geom* g, const double* xyz_host, int64_t T, void* stream, sbio_targets** out);
int sbio_targets_destroy(sbio_targets* ts);
/* Points, near (point, spheroid) pairs, far (point, source node) pairs and
 * device bytes of the set (outputs may be NULL). */
int sbio_targets_info(const sbio_targets* ts, int64_t* n_points, int64_t* n_near_pairs, int64_t* n_far_pairs,
                      size_t* device_bytes);
/* S_out[t] = S[sigma](x_t), D_out[t] = D[mu](x_t): inputs as
 * sbio_apply_laplace (device, M x (p+1)^2, either may be NULL), outputs
 * device arrays of T doubles, overwritten.  Precision and far-field launch
 * shape are the geometry's.  Uses the geometry's workspaces: stream-ordered
 * with every other call on the same geometry.  Asynchronous. */
int sbio_eval_targets(sbio_targets* ts, const double* sigma_tilde, const double* mu_hat, double* S_out,
                      double* D_out, void* stream);

/* Directional derivatives of the layer potentials at the set's points
 * (Sec. 3.3, Theorem 3 and eq. (dSLevalformula), with the particle-to-target
 * split of Sec. 4.1): Sp_out[t] = grad S[sigma](x_t) . e_t and
 * Dp_out[t] = grad D[mu](x_t) . e_t, e_t = dirs[3t .. 3t+2] (device, T x 3
 * FP64, taken as given: not normalised).  Near pairs differentiate the
 * source's exterior expansions (at a point on a surface this is the exterior
 * limit: S'+ = S' - sigma/2 of sbio_apply_laplace_deriv); far pairs the
 * differentiated quadrature.  Inputs and outputs as sbio_eval_targets (either
 * density may be NULL; each output is given exactly when its input is;
 * outputs overwritten).  SBIO_ENOTSUP for p > 20.  Asynchronous. */
int sbio_eval_targets_deriv(sbio_targets* ts, const double* dirs, const double* sigma_tilde, const double* mu_hat,
                            double* Sp_out, double* Dp_out, void* stream);

/* Stokes single layer (viscosity 1) at the set's points (Sec. 4.3 with the
 * particle-to-target algorithm): u_out (device, T x 3) = S_stk[f](x_t) by
 * eq. (stokes) for near pairs and the Stokeslet quadrature otherwise;
 * p_out (device, T, may be NULL) = the pressure with the printed kernel
 * P = r / (4 pi |r|^3), i.e. -sum_j d_j S[f_j] for near pairs (the printed
 * identity in terms of gradients of S has the opposite sign).  f_tilde as in
 * sbio_apply_stokes_sl.  Outputs overwritten; SBIO_ENOTSUP for p > 20;
 * stream-ordered with the geometry's other calls.  Asynchronous. */
int sbio_eval_targets_stokes(sbio_targets* ts, const double* f_tilde, double* u_out, double* p_out, void* stream);

/* Stokes double layer (as sbio_apply_stokes_dl) at the set's points: u_out
 * device T x 3, overwritten.  SBIO_ENOTSUP for p > 20.  Asynchronous. */
int sbio_eval_targets_stokes_dl(sbio_targets* ts, const double* q_hat, double* u_out, void* stream);


/* ---- forward transform and exterior boundary-value solves (Sec. 2.3,
 * Sec. 5.1) -----------------------------------------------------------------
 * Forward transform: coefficients of node values f (device, N, the node
 * layout of the outputs), f^_nm = sum_j w_j (2 pi / n_phi) sum_k f_jk Y_nm,
 * exact for band-limited f of degree <= p; modified != 0 gives the
 * modified-basis coefficients (those of f sqrt(u0^2 -+ v^2), Sec. 3.2).
 * coef_out: device, M x (p+1)^2.  Asynchronous. */
int sbio_forward_transform(sbio_geom* g, const double* values, int32_t modified, double* coef_out, void* stream);

/* Completion terms of the Dirichlet formulation (Sec. 5.1): C_I places at
 * each centre a charge equal to int sigma_i dS with kernel 1/|x - c_i| (as
 * printed, no 1/(4 pi)); S adds the single layer of the same density; the
 * ETA forms scale particle i's term by eta_i from the paper's table of
 * heuristic scalings (eps = 1/aspect ratio; C_I: eps / area of the spheroid
 * with major semi-axis 1, 0.06 for oblates with aspect ratio > 3; S: prolate
 * 0.5 or 1/(2 eps log(1/eps)) above aspect ratio 3, oblate 1/(4 eps) + 1/4 or
 * 1 above 3). */
#define SBIO_COMPLETION_CI 0
#define SBIO_COMPLETION_ETA_CI 1
#define SBIO_COMPLETION_S 2
#define SBIO_COMPLETION_ETA_S 3

typedef struct {
  int32_t iterations;   /* Arnoldi steps (operator applications, not counting residual checks) */
  int32_t restarts;     /* completed restart cycles that had not converged */
  int32_t converged;    /* 1 if the true relative residual reached tol */
  double rel_residual;  /* ||b - K x|| / ||b|| at exit (coefficient space) */
  double ms;            /* wall time of the call */
} sbio_solve_info;

/* Exterior Dirichlet problem with the completed double layer: finds sigma
 * with 1/2 sigma + D[sigma] + C[sigma] = f on every surface, so that
 * u = D[sigma] + C[sigma] solves it in the fluid.  Solved in coefficient
 * space (unknown: the plain coefficients of sigma; operator: the forward
 * transform of the node values of D + C; right-hand side: the transform of
 * f) by restarted GMRES(restart) from zero to relative residual tol, at most
 * max_iter Arnoldi steps.  f_nodes: device, N.  Outputs (device): mu_hat_out
 * M x (p+1)^2 = sigma's coefficients; sigma_tilde_out (M x (p+1)^2, may be
 * NULL) = modified coefficients of the S completion term (zeros for C_I),
 * charges_out (M, may be NULL) = the C_I charges (zeros for S), so that
 * u(x) = D[mu_hat](x) + S[sigma_tilde](x) + sum_i charges_i/|x - c_i| (the
 * first two through sbio_eval_targets).  Uses the geometry's precision and
 * workspaces; allocates its Krylov basis ((restart+1) M (p+1)^2 doubles,
 * stream-ordered, charged to the context budget: SBIO_ENOMEM); synchronises
 * `stream` (the iteration is driven from the host).  info may be NULL;
 * non-convergence is reported in info, not as an error.  In SBIO_MIXED the
 * operator carries the far field's FP32 rounding (about 1e-7 relative), which
 * bounds the reachable residual: use tol >= 1e-6 there. */
int sbio_solve_dirichlet(sbio_geom* g, const double* f_nodes, int32_t completion, double tol, int32_t max_iter,
                         int32_t restart, double* mu_hat_out, double* sigma_tilde_out, double* charges_out,
                         sbio_solve_info* info, void* stream);

/* Exterior Neumann problem with the single layer: finds rho with
 * -1/2 rho + S'[rho] = g on every surface (u = S[rho]); unknown and output
 * rho_tilde_out: device, M x (p+1)^2 modified coefficients (the input
 * convention of the S apply); right-hand side g_nodes: device, N (the outward
 * normal derivative of u).  As sbio_solve_dirichlet otherwise; SBIO_ENOTSUP
 * for p > 20. */
int sbio_solve_neumann(sbio_geom* g, const double* g_nodes, double tol, int32_t max_iter, int32_t restart,
                       double* rho_tilde_out, sbio_solve_info* info, void* stream);

/* ---- batched apply over many suspensions ------------------------------
 * A batch groups resident geometries (any mix of M and p, all in SBIO_MIXED
 * mode, same context).  One batch apply computes S[sigma_s] and D[mu_s] for
 * every suspension s as one CUDA graph: the synthesis/self kernels, the
 * near-field kernels on a second branch, and a single persistent far-field
 * kernel whose CTAs pull (suspension, target block, source-tile range) work
 * items from an atomic counter, longest first.  No data is shared between
 * suspensions (they are independent problems).  The graph is captured on the
 * first apply and replayed while the same buffers are passed; new buffers
 * trigger a re-capture (which synchronises `stream`).  A geometry whose far
 * field is the treecode (sbio_geom_set_far_method, set before
 * sbio_batch_create) has its treecode kernels in the graph on the near
 * branches instead of items of the persistent kernel. */
typedef struct sbio_batch sbio_batch;

/* geoms: host array of n geometry handles, kept alive by the caller until
 * sbio_batch_destroy.  Errors: SBIO_EINVAL (null, other context, FP64 mode). */
int sbio_batch_create(sbio_ctx* ctx, sbio_geom* const* geoms, int32_t n, sbio_batch** out);
int sbio_batch_destroy(sbio_batch* b);

/* Work items, total far pairs per apply, targets per thread of the far
 * kernel and its persistent grid size (outputs may be NULL). */
int sbio_batch_info(const sbio_batch* b, int64_t* n_items, int64_t* far_pairs, int32_t* far_tt, int32_t* grid);

/* Targets per thread (1, 2, 4, 8, or -2, -4, -8 for the packed f32x2 form) of
 * the persistent far kernel; rebuilds the
 * work list and drops the captured graph. */
int sbio_batch_set_far_tt(sbio_batch* b, int32_t far_tt);

/* sigma, mu, S_out, D_out: host arrays of n device pointers (layouts as in
 * sbio_apply_laplace for each suspension).  Asynchronous on `stream`. */
/* Autotuner of a batch (the launch shapes are the library's to choose, the
 * tuner the project writes): times whole batched steps (CUDA events on
 * `stream`, best of two after one warm replay, graph recaptured per shape)
 * over the persistent far kernel's targets per thread (1, 2, 4, 8 scalar;
 * 2, 4, 8 packed), then the near kernels' thread-group size (64 or 128
 * threads per CTA, set on every geometry of the batch), then the persistent
 * grid (2, 3, 4, 5, 6 or 8 CTAs per SM; below 4 the near kernels of the
 * graph's other branch find free SM slots beside it), keeps the fastest and
 * reports it (any
 * output may be NULL; step_ms is its step time).  The buffers are those of
 * sbio_batch_apply and are overwritten.  Synchronises `stream`. */
int sbio_batch_autotune(sbio_batch* b, const double* const* sigma, const double* const* mu, double* const* S_out,
                        double* const* D_out, void* stream, int32_t* far_tt, int32_t* near_block,
                        int32_t* ctas_per_sm, double* step_ms);

int sbio_batch_apply(sbio_batch* b, const double* const* sigma, const double* const* mu,
                     double* const* S_out, double* const* D_out, void* stream);

/* ---- request serving with continuous batching ----------------------------
 * A server owns n_slots worker threads, each with its own CUDA stream, and a
 * device-memory budget.  Requests are admitted first-in first-out as soon as
 * a slot is free and the request's estimated footprint fits the budget (a
 * request that does not fit waits until running ones release memory; a lone
 * request is always admitted).  An admitted request builds its geometry once,
 * runs n_applies applies with fresh coefficients while geometry and near
 * lists stay resident, writes every result to its host buffer and releases the
 * geometry.  Work of different slots overlaps on the device. */
#define SBIO_OP_LAPLACE 0   /* S[sigma] and D[mu] (sbio_apply_laplace) */
#define SBIO_OP_STOKES 1    /* Stokes single layer (sbio_apply_stokes_sl) */

typedef struct sbio_server sbio_server;

/* One request.  coef_host: n_applies consecutive coefficient sets in host
 * memory (Laplace: sigma~ then mu^, 2 x M x (p+1)^2 each; Stokes: M x 3 x
 * (p+1)^2 each).  out_host: n_applies consecutive results (Laplace: S then D,
 * 2 x N each; Stokes: N x 3 each).  Both buffers stay owned by the caller and
 * must stay valid until sbio_server_wait returns for the ticket; sph is copied
 * at submission. */
#define SBIO_REQ_TREE 1u  /* request flag: far field by the treecode (order 16, theta 0.5;
                             mixed-precision requests with at least 50,000 nodes,
                             see sbio_geom_set_far_method; smaller ones stay direct) */

typedef struct {
  int32_t op;
  int32_t n_applies;
  const sbio_spheroid* sph;
  int32_t M;
  int32_t flags;   /* 0 or SBIO_REQ_TREE */
  sbio_options opts;
  const double* coef_host;
  double* out_host;
} sbio_request;

/* mem_budget_bytes = 0: no budget.  The server's geometries belong to ctx. */
int sbio_server_create(sbio_ctx* ctx, int32_t n_slots, size_t mem_budget_bytes, sbio_server** out);

/* Validates and queues a request; returns its ticket. */
int sbio_server_submit(sbio_server* s, const sbio_request* r, int64_t* ticket);

/* Waits at most timeout_s seconds for a ticket (SBIO_ETIMEOUT if not done; the
 * ticket stays valid).  status: 0 or the request's error code; latency_ms:
 * submission to last result on the host; service_ms: admission to last result.
 * A ticket can be waited for successfully once. */
int sbio_server_wait(sbio_server* s, int64_t ticket, double timeout_s, int32_t* status, double* latency_ms,
                     double* service_ms);

/* Completed requests and applies so far, running and queued requests, device
 * bytes currently reserved by admitted requests (outputs may be NULL). */
int sbio_server_stats(sbio_server* s, int64_t* completed, int64_t* applies, int32_t* running, int32_t* queued,
                      size_t* reserved);

/* Drains the queue (every submitted request runs), joins the workers and
 * releases the server. */
int sbio_server_destroy(sbio_server* s);

/* Allocation-free self interaction (no counterpart in the paper; a service for
 * callers that cannot allocate device memory).
 *
 * Computes the on-surface self part only -- for each spheroid, S and D of its
 * own density at its own nodes (the diagonal multipliers of Theorems 1-2
 * followed by the inverse transform, i.e. the block-diagonal part of
 * sbio_apply_laplace) -- without creating a geometry and without calling
 * cudaMalloc, cudaFree or any allocating routine.  It is meant for code that
 * must not allocate: a solver running inside a framework whose allocator or
 * start-up reservation already owns the device memory (a private cudaMalloc
 * could fail or fragment that pool), or a loop that was promised never to
 * allocate after initialisation.  The caller passes its own device buffers:
 *   sph: host array of M descriptors; p, n_phi as in sbio_options (n_phi 0 =
 *        2(p+1)); sigma_tilde / mu_hat: device, M x (p+1)^2 (either may be
 *        NULL); S_out / D_out: device, N (given exactly when the matching
 *        input is).  Outputs are overwritten; asynchronous on `stream`.
 * All other device data lives in one fixed array of 8 MiB that every GPU
 * holding the library's module keeps reserved until the process exits.  A
 * request whose tables and workspaces do not fit (about 80 spheroids at
 * p = 16) fails with SBIO_EINVAL before any device work.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array: calls whose GPU
 * work overlaps (other streams, other host threads) race and must be
 * serialised by the caller.  Nothing in the array needs to start at zero.
 * The tables are staged from a host buffer that is freed when the call
 * returns, so a call on a stream that is being captured fails with
 * SBIO_EINVAL. */
int sbio_apply_self_noalloc(const sbio_spheroid* sph, int32_t M, int32_t p, int32_t n_phi,
                            const double* sigma_tilde, const double* mu_hat, double* S_out,
                            double* D_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SBIO_H */
