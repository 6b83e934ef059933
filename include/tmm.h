/*
 * tmm.h -- C ABI of libtmm, a GB300 (sm_103a) library for the batched
 * coherent transfer-matrix method of TMM-Fast (arXiv 2111.13667).
 *
 * Physics (arXiv 2111.13667, Sec. 2): a plane wave of vacuum wavelength
 * lambda enters a stack from the semi-infinite injection medium 0 at angle
 * theta, crosses L finite layers (index n_j, thickness d_j) and leaves into
 * the semi-infinite outcoupling medium L+1.  For every (stack, lambda, theta,
 * polarisation) the library evaluates Snell's law, the Fresnel coefficients
 * of Eq. 1, the layer matrices of Eq. 3, their product (Eq. 4), the
 * extraction of r and t (Eqs. 5-6) and R, T (Eq. 2).
 *
 * Conventions shared by every entry point
 *   - Time dependence exp(-i omega t); absorbing media have n = n' + i k with
 *     k >= 0.  Lengths in nm, angles in radians in medium 0.
 *   - Complex arrays are interleaved (re, im) pairs of the working type.
 *   - Root of cos(theta_j): the one whose n_j cos(theta_j) has a positive
 *     imaginary part (decaying along +z); if that part is zero to rounding,
 *     the one with positive real part.  Im(delta_j) of a layer's phase is
 *     clamped at 35 (opaque layers).  At exact grazing incidence
 *     (cos(theta_0) = 0) R = 1 and T = 0.  T follows the Poynting-flux form of
 *     Eq. 2: s: Re(n_out c_out)/Re(n_in c_in)|t|^2, p: with conj(c).
 *   - Every pointer named "device" is caller-owned device memory, contiguous,
 *     C order, in the working type selected by `prec` (double for TMM_F64,
 *     float for TMM_F32) unless stated otherwise.  The library keeps no
 *     pointer after a call returns and allocates no device memory, except the
 *     surrogate object, which owns its weights.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Arguments are checked on the host
 *     before anything is launched; a rejected call launches nothing.  No C++
 *     exception crosses this boundary.
 *   - Values that can only be checked on the device (a material index out of
 *     range, a layer count outside [0, L_max], a complex injection index)
 *     poison the outputs of the affected stack with NaN instead of reading
 *     out of bounds.
 *   - Host threads: the library's host-side caches (device facts, each
 *     kernel's shared-memory limit) are guarded by locks, and a kernel's
 *     limit only ever grows, so calls may come from several host threads at
 *     once, each with its own stream and buffers.  Two exceptions share state
 *     across calls: tmm_coh_batched_noalloc (one scratch array, see there) and
 *     tmm_gemm_bf16(_t), which report an expired pipeline wait through one
 *     flag per device, so concurrent calls of those can attribute a timeout
 *     to the wrong call.  Each surrogate object has its own flag; calls on one
 *     object are ordered by their stream.
 */
#ifndef TMM_GB300_TMM_H
#define TMM_GB300_TMM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TMM_API __attribute__((visibility("default")))
#else
#define TMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TMM_OK = 0,
    TMM_ERR_INVALID_ARG = -1, /* a host-side argument check failed */
    TMM_ERR_UNSUPPORTED = -2, /* valid request this build cannot serve */
    TMM_ERR_CUDA = -3,        /* a CUDA runtime call failed (see tmm_last_cuda_error) */
    TMM_ERR_TIMEOUT = -4,     /* a device-side iteration limit was hit */
    TMM_ERR_NOMEM = -5        /* workspace too small / host allocation failed */
} tmm_status;

/*
 * TMM_F64   native FP64 arithmetic, double arrays.
 * TMM_F32   FP32 arithmetic, float arrays.
 * TMM_F64X  double arrays, double-float arithmetic (each value the unevaluated
 *           sum of two floats, ~48 significant bits) on the FP32 pipes: the
 *           FP64 tolerance at several times the native FP64 throughput of this
 *           part.  Forward only (tmm_coh_batched / _ex, non-persistent).
 * TMM_F32D  FP32 arithmetic on double inputs: n_direct / mat_table, d, theta
 *           and lambda are double (as for TMM_F64), R and T are float.  The
 *           per-(layer, wavelength) part of each layer phase is formed from
 *           the double values, so rounding the inputs to float costs nothing;
 *           the FP32 result then holds the FP32 tolerance also where the
 *           stack magnifies input rounding (thick resonant stacks near
 *           grazing incidence).  Forward only (tmm_coh_batched / _ex,
 *           persistent or not, and tmm_coh_batched_noalloc); every other entry
 *           point returns TMM_ERR_UNSUPPORTED.
 *
 * FP32 layer phase (TMM_F32 and TMM_F32D): the phase of layer j in turns,
 * (d_j / lambda) Re q_j with q_j = n_j cos(theta_j), is evaluated as
 * (d_j / lambda) Re n_j -- angle-independent, staged per (layer, wavelength)
 * in double-float arithmetic -- plus (d_j / lambda) Re(q_j - n_j), where
 * q_j - n_j = -beta^2 / (q_j + n_j) by Snell's law (beta = n_0 sin theta):
 * float roundings act only on the angle-dependent part of the phase.
 */
typedef enum { TMM_F64 = 0, TMM_F32 = 1, TMM_F64X = 2, TMM_F32D = 3 } tmm_prec;

/* Polarisation bits of tmm_problem.pol_mask; outputs store s before p.
 * TMM_POL_AVG, only together with both TMM_POL_S and TMM_POL_P (pol_mask 7),
 * writes one plane holding (R_s + R_p) / 2 and (T_s + T_p) / 2: unpolarised
 * light, as the paper averages s and p for its reflectivity map (Fig. 2). */
#define TMM_POL_S 1u
#define TMM_POL_P 2u
#define TMM_POL_AVG 4u

/*
 * One batched problem: S stacks, each with up to L_max finite layers,
 * evaluated on an n_lambda x n_theta grid for the polarisations in pol_mask.
 *
 * The complex index of medium j of stack s at wavelength l comes from exactly
 * one of two sources (index assembly; Sec. 3, coh_tmm_fast / _disp, and the
 * material matrix I of Sec. 5):
 *   direct:    n_direct != NULL.  n_direct_per_lambda = 1: complex
 *              [S][L_max+2][n_lambda]; = 0: complex [S][L_max+2] (no
 *              dispersion).  mat_table, mat_idx must be NULL.
 *   gathered:  mat_table complex [n_materials][n_lambda] and mat_idx int32
 *              [S][L_max+2] (device); n[s][j][l] = mat_table[mat_idx[s][j]][l].
 * Media rows hold 0 (injection), 1..L_s (finite layers) and L_s+1
 * (outcoupling); Im(n_0) must be 0.
 *   d            device [S][L_max]: thickness of finite layer j at d[s][j-1].
 *   L_per_stack  device int32 [S] or NULL.  NULL: every stack has L_max
 *                layers.  Otherwise stack s has L_s layers (0 <= L_s <=
 *                L_max); its rows past L_s+1 and thicknesses past L_s are
 *                never read.
 *   theta        device [n_theta], radians in medium 0.
 *   lambda       device [n_lambda], vacuum wavelength in nm.
 */
typedef struct {
    int32_t S, L_max, n_lambda, n_theta;
    uint32_t pol_mask; /* TMM_POL_S | TMM_POL_P */
    int32_t prec;      /* tmm_prec */
    const void *n_direct;
    int32_t n_direct_per_lambda;
    const void *mat_table;
    const int32_t *mat_idx;
    int32_t n_materials;
    const void *d;
    const int32_t *L_per_stack;
    const void *theta;
    const void *lambda;
} tmm_problem;

/*
 * Launch shape (all fields 0 = library default).  One block evaluates one
 * work item: one stack x tile_lambda wavelengths x tile_theta angles, each
 * thread covering the requested polarisations.  FP32 and double-float tiles
 * of two or more angles run two adjacent angles per thread (the two lanes of
 * the paired FP32 instructions): tile_lambda x ceil(tile_theta / 2) threads,
 * at most 256; otherwise one (lambda, theta) per thread, at most 512.
 *   persistent   0: one block per work item.  1: a persistent grid pulls work
 *                items from a device counter, longest stacks first (ragged
 *                batches); needs a workspace (tmm_workspace_size).
 *   blocks_per_sm  persistent grid size = blocks_per_sm x SM count.
 *   max_items_per_block  persistent only: a block that has taken this many
 *                items stops, flags TMM_ERR_TIMEOUT in the workspace and
 *                returns (0 = no limit beyond the item count).
 */
typedef struct {
    int32_t tile_lambda;
    int32_t tile_theta;
    int32_t persistent;
    int32_t blocks_per_sm;
    int32_t max_items_per_block;
} tmm_launch_cfg;

/*
 * R and T for every (pol, stack, theta, lambda) (Sec. 2, Eqs. 1-6).
 *   R  device [P][S][n_theta][n_lambda], P = number of polarisation bits in
 *      pol_mask (s, p), or 1 with TMM_POL_AVG
 *   T  same layout, or NULL to skip it
 * Equivalent to tmm_coh_batched_ex with the default launch shape and no
 * workspace.
 */
TMM_API tmm_status tmm_coh_batched(const tmm_problem *p, void *R, void *T, void *stream);

/*
 * As tmm_coh_batched with an explicit launch shape (cfg may be NULL).  A
 * persistent launch needs `workspace` (device, at least the bytes reported by
 * tmm_workspace_size, 256-byte aligned); the call zeroes what it uses.  The
 * whole call is a fixed sequence of launches and memsets on `stream`, so it
 * can be captured in a CUDA graph.
 */
TMM_API tmm_status tmm_coh_batched_ex(const tmm_problem *p, const tmm_launch_cfg *cfg,
                              void *workspace, size_t workspace_bytes, void *R, void *T,
                              void *stream);

/*
 * R and T (Sec. 2, Eqs. 1-6) for a problem whose arrays live in HOST memory:
 * the call copies the inputs to the device, evaluates the stacks in n_chunks
 * contiguous chunks on `stream`, and copies every chunk's R and T back while
 * the next chunks run (three device slots of chunk outputs; the copies go on
 * a stream of their own).  Only the last chunk's copy is exposed.
 *   p          as for tmm_coh_batched, but every array pointer is host memory
 *              (page-locked memory lets the copies overlap the kernels;
 *              pageable memory works, serialised); prec TMM_F64, TMM_F32,
 *              TMM_F32D or TMM_F64X
 *   R, T       host [P][S][n_theta][n_lambda] of the output type (T may be NULL)
 *   n_chunks   1 .. S (else TMM_ERR_INVALID_ARG)
 *   workspace  device, >= tmm_host_workspace_size(p, n_chunks) bytes,
 *              256-byte aligned: the inputs' device copies and the output slots
 * Asynchronous on `stream` like the other entry points: the host inputs must
 * stay unchanged, and R, T are complete, only once `stream` has synchronised.
 * The call creates and releases one stream and a few events of its own.
 * Calls that share a workspace must be serialised by the caller.
 */
TMM_API tmm_status tmm_host_workspace_size(const tmm_problem *p, int32_t n_chunks, size_t *bytes);
TMM_API tmm_status tmm_coh_batched_host(const tmm_problem *p, int32_t n_chunks, void *workspace,
                                        size_t workspace_bytes, void *R, void *T, void *stream);

/* Workspace bytes tmm_coh_batched_ex / tmm_coh_grad need for this problem. */
TMM_API tmm_status tmm_workspace_size(const tmm_problem *p, const tmm_launch_cfg *cfg,
                              size_t *bytes);

/*
 * Status a persistent launch recorded in its workspace: TMM_OK or
 * TMM_ERR_TIMEOUT.  Synchronises `stream`.
 */
TMM_API tmm_status tmm_workspace_status(const void *workspace, void *stream);

/*
 * Per-stack merit and its adjoint gradient (replaces the autograd path of
 * Sec. 4 / appendix A.3):
 *   merit[s] = mean over (pol, theta, lambda) of (R - R_target)^2
 *   dm_dd[s][j-1] = d merit[s] / d d_j                      (1/nm)
 *   dm_dn[s][j-1] = d merit[s] / d (Delta n_j), where n_j(lambda) ->
 *                   n_j(lambda) + Delta n_j (a real offset at every lambda);
 *                   for a non-dispersive index this is d merit / d n_j.
 * Entries past L_s are written as 0.
 *   R_target  device [P][n_theta][n_lambda] (shared by every stack)
 *   merit     device [S]; dm_dd device [S][L_max]; dm_dn device [S][L_max] or NULL
 *   workspace optional: with a workspace of tmm_workspace_size(p, NULL)
 *             bytes each stack is split over several blocks and reduced in a
 *             fixed order in a second pass; with NULL one block covers a
 *             stack.  Results are deterministic either way.
 */
TMM_API tmm_status tmm_coh_grad(const tmm_problem *p, const void *R_target, void *merit,
                        void *dm_dd, void *dm_dn, void *workspace, size_t workspace_bytes,
                        void *stream);

/*
 * Stacks with incoherent (thick) layers.  The paper treats coherent stacks
 * only; this extends tmm_coh_batched in the usual way: media 0 and L_s+1 and
 * every finite layer flagged in `incoherent` are incoherent; the coherent
 * blocks between consecutive incoherent media are evaluated as amplitude
 * products (Eqs. 1-6) and combined through the incoherent layers by
 * intensities (each block's R and T for light from either side).
 *   incoherent  device uint8 [S][L_max], nonzero = incoherent layer; NULL =
 *               none (the coherent result)
 *   R, T        as tmm_coh_batched (T may be NULL); pol_mask 1, 2, 3 or 7
 * An incoherent layer may absorb: each single pass of light through it is
 * attenuated by exp(-4 pi Im(n_j cos theta_j) d_j / lambda) (Beer-Lambert
 * along the refracted path), and the blocks next to it see its complex index
 * in their Fresnel coefficients and Poynting factors.  The first incoherent
 * layer with Re(n_j^2 - n_0^2 sin^2 theta) <= 0 (for a real index: the wave
 * is evanescent) ends the stack: it is the exit medium for R and T = 0.  prec
 * TMM_F64 or TMM_F32 (else TMM_ERR_UNSUPPORTED).  Asynchronous on `stream`.
 */
TMM_API tmm_status tmm_inc_batched(const tmm_problem *p, const uint8_t *incoherent, void *R, void *T,
                                   void *stream);

/*
 * Absorbed fraction of the incident power in every layer, from the partial
 * products of Eq. 4 (the paper notes partial coefficients come from
 * multiplying only part of the chain): A_j = F_j - F_{j+1}, F_j the Poynting
 * flux at the left boundary of layer j normalised by the incident flux
 * (F_1 = 1 - R, F_{L+1} = T, so R + T + sum_j A_j = 1).
 *   A     device [P][S][L_max][n_theta][n_lambda]; entries j >= L_s are 0;
 *         with TMM_POL_AVG one plane holding (A_s + A_p) / 2
 *   R, T  device [P][S][n_theta][n_lambda] from the same sweep, or NULL (T
 *         may be NULL alone)
 * Limits: L_max <= 127 (else TMM_ERR_UNSUPPORTED); prec TMM_F64 or TMM_F32.
 * Exact grazing incidence gives A = 0, R = 1, T = 0.  Asynchronous on `stream`.
 */
TMM_API tmm_status tmm_absorption_batched(const tmm_problem *p, void *A, void *R, void *T, void *stream);

/*
 * Field intensity inside every layer: |E(z) / E_inc|^2 at the depths
 * z_k = (k + 1/2) d_j / n_z, k = 0 .. n_z - 1, of every layer j, from the same
 * partial products (E_inc: the incident plane wave's field amplitude; for p
 * both the tangential and the normal field component count).
 * k0 Im(n_j^2) |E|^2 |E_inc|^2 is the absorption density whose integral over
 * layer j is tmm_absorption_batched's A_j times the incident flux.
 *   E    device [P][S][L_max][n_z][n_theta][n_lambda]; layers j >= L_s are 0;
 *        with TMM_POL_AVG one plane of the mean of s and p
 * Limits: n_z >= 1 (else TMM_ERR_INVALID_ARG); prec TMM_F64 or TMM_F32; one
 * wavelength's staged stack, (L_max + 2) x 6 reals, must fit in shared memory
 * (L_max up to about 4800 in FP64), else TMM_ERR_UNSUPPORTED.  Exact grazing
 * incidence gives 0.  Asynchronous on `stream`.
 */
TMM_API tmm_status tmm_field_profile(const tmm_problem *p, int32_t n_z, void *E, void *stream);

/*
 * One partially coherent layer per stack (the paper treats coherent stacks
 * only; this is a reading of partial coherence as a Gaussian spread of one
 * layer's thickness, from nonuniformity or a finite coherence length).
 * Finite layer j = layer[s] (1-based; 0 = a coherent stack) has the thickness
 * d_j + D, D ~ N(0, sigma[s]^2) nm, and R, T are the expectations of the
 * coherent R, T (Eqs. 1-6) over D, by the Gauss-Hermite rule with n_nodes
 * nodes x_k and weights w_k: E[f] = sum_k (w_k / sqrt(pi)) f(sqrt(2) sigma x_k).
 * A node whose thickness falls below zero counts as zero thickness.
 *   layer    device int32 [S]
 *   sigma    device real [S] (the problem's real type), nm
 *   n_nodes  1 .. 256 (else TMM_ERR_INVALID_ARG).  The rule resolves fringe
 *            harmonics up to a frequency growing like sqrt(n_nodes): phase
 *            spreads 2 pi Re(n_j cos theta_j) sigma / lambda of about 1 need
 *            some 30 nodes, of about 2 some 250; wider spreads are the
 *            incoherent limit (tmm_inc_batched)
 *   R, T     device [P][S][n_theta][n_lambda] as tmm_coh_batched (T may be
 *            NULL; TMM_POL_AVG gives one plane of the mean of s and p)
 * A stack whose layer is outside [0, L_s] or whose sigma is negative or not
 * finite gets NaN.  prec TMM_F64 or TMM_F32 (else TMM_ERR_UNSUPPORTED); the
 * stage limit on L_max of tmm_field_profile.  Asynchronous on `stream`.
 */
TMM_API tmm_status tmm_pcoh_batched(const tmm_problem *p, const int32_t *layer, const void *sigma, int32_t n_nodes,
                                    void *R, void *T, void *stream);

/*
 * Batched reward of the paper's reinforcement-learning environment (Sec. 5):
 *   reward[s] = - sum over (plane, theta, lambda) of |R_target - R|
 * for every stack, with the planes of pol_mask (s, p, or their mean for
 * TMM_POL_AVG).  The forward kernels run in a reduction mode: no R or T is
 * written; each (stack, tile) work item leaves its partial sum in the
 * workspace and a second pass adds them in a fixed order (deterministic).
 * Ragged stacks (L_per_stack) and the persistent longest-first launch work
 * as for tmm_coh_batched_ex (cfg->max_items_per_block must be 0 here).
 *   R_target   device [P][n_theta][n_lambda]
 *   reward     device [S], the real type of p->prec (F32 or F64; F64X:
 *              TMM_ERR_UNSUPPORTED)
 *   workspace  device, >= tmm_reward_workspace_size(p, cfg) bytes, 256-byte
 *              aligned, caller-owned scratch
 * Asynchronous on `stream`.
 */
TMM_API tmm_status tmm_reward_workspace_size(const tmm_problem *p, const tmm_launch_cfg *cfg, size_t *bytes);
TMM_API tmm_status tmm_coh_reward(const tmm_problem *p, const tmm_launch_cfg *cfg, const void *R_target,
                                  void *reward, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Merit-driven thickness optimisation: the use case of the paper's Fig. 1c
 * (a merit of R over wavelength and angle minimised over the thicknesses with
 * the gradients of Sec. 4).  The paper fixes no optimiser; this runs Adam
 * (Kingma and Ba, 2015) on every stack at once, each stack an independent
 * start.  One step evaluates merit and dm/dd exactly as tmm_coh_grad does at
 * the current thicknesses, then updates every finite layer j < L_s:
 *   m = beta1 m + (1 - beta1) g,   v = beta2 v + (1 - beta2) g^2,
 *   d = clip(d - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps),
 *            d_min, d_max)
 * with t = step0 + 1, step0 + 2, ...  Layers past L_s keep their values.
 *   p           the problem; p->d (device [S][L_max], the real type of
 *               p->prec) is READ AND OVERWRITTEN in place.  prec TMM_F64 or
 *               TMM_F32 (TMM_F64X: TMM_ERR_UNSUPPORTED).
 *   R_target    device [P][n_theta][n_lambda], as for tmm_coh_grad
 *   cfg         host: lr > 0, 0 <= beta1, beta2 < 1, eps > 0,
 *               d_min <= d_max (nm); step0 >= 0 = steps already taken with
 *               this workspace (0 resets the moment estimates m, v)
 *   steps       >= 0 Adam steps in this call
 *   merit_hist  device [steps][S] or NULL: merit at the start of each step
 *   workspace   device, >= tmm_optimize_workspace_size bytes, 256-byte
 *               aligned, caller-owned; keeps m and v between calls
 * Asynchronous on `stream`; argument errors are returned before any launch.
 */
typedef struct {
    double lr, beta1, beta2, eps, d_min, d_max;
    int32_t step0;
    int32_t reserved; /* 0 */
} tmm_adam_cfg;

TMM_API tmm_status tmm_optimize_workspace_size(const tmm_problem *p, size_t *bytes);
TMM_API tmm_status tmm_optimize_adam(const tmm_problem *p, const void *R_target, const tmm_adam_cfg *cfg,
                                     int32_t steps, void *merit_hist, void *workspace,
                                     size_t workspace_bytes, void *stream);

/* Short description of a status code (static string). */
TMM_API const char *tmm_status_string(int status);

/* Message of the last CUDA error this library saw on the calling thread. */
TMM_API const char *tmm_last_cuda_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
TMM_API int32_t tmm_version(void);

/*
 * Issue-rate probe, not part of the method: runs independent FMA chains in
 * the working type on every SM and reports the achieved rate.
 *   flops_per_s  host out: 2 x FMAs per second;  ms  host out: kernel time.
 * Synchronises `stream`.
 */
TMM_API tmm_status tmm_probe_fma_rate(int32_t prec, double *flops_per_s, float *ms, void *stream);

/*
 * Learned surrogate (motivated by the paper's dataset generation for machine
 * learning, abstract and Sec. "Core functionality speedup and dataset
 * generation"; the network itself is not in the paper): an MLP from the L
 * thicknesses of a fixed stack to its R spectra, s then p, theta-major,
 * lambda fastest (2 n_theta n_lambda outputs).  Hidden layers of width
 * `hidden` with GELU (erf form), a linear head; bf16 weights and activations,
 * fp32 accumulation on the tcgen05 tensor cores; Adam on fp32 masters.  The
 * exact transfer-matrix kernel (FP32) generates training spectra and judges
 * inference outputs.  The object owns its device memory (weights, optimizer
 * state, batch buffers grown on demand; growth synchronises the device).
 */
typedef struct tmm_surrogate tmm_surrogate;
typedef struct {
    int32_t n_layers;        /* L finite layers, 1..64 */
    const double *n_media;   /* host complex [L+2] (re, im): media 0..L+1; Im n_0 = 0 */
    int32_t n_lambda;
    const double *lambda;    /* host [n_lambda], nm */
    int32_t n_theta;
    const double *theta;     /* host [n_theta], radians */
    double d_min, d_max;     /* thickness range; inputs are mapped to [0, 1] */
    int32_t hidden;          /* width, multiple of 64 */
    int32_t depth;           /* hidden layers, 1..16 */
    uint64_t seed;           /* weight initialisation */
} tmm_surrogate_desc;

TMM_API tmm_status tmm_surrogate_create(const tmm_surrogate_desc *desc, tmm_surrogate **out);
TMM_API void tmm_surrogate_destroy(tmm_surrogate *s);
TMM_API int32_t tmm_surrogate_outputs(const tmm_surrogate *s);
TMM_API int64_t tmm_surrogate_parameters(const tmm_surrogate *s);
/* Exact spectra (training targets): d device [B][L] f32 -> R device [B][outputs] f32. */
TMM_API tmm_status tmm_surrogate_generate(tmm_surrogate *s, const float *d, int32_t B, float *R, void *stream);
/* One Adam step on the MSE between the network and R_target (device [B][outputs]);
 * B a multiple of 8, >= 128; loss: device f32 (mean squared error) or NULL. */
TMM_API tmm_status tmm_surrogate_train_step(tmm_surrogate *s, const float *d, const float *R_target, int32_t B,
                                            float lr, float *loss, void *stream);
/* R device [B][outputs] = clamp(network(d), 0, 1).  Every round(1/judge_fraction)-th
 * row (judge_fraction in [0, 1]; 0 = none, 1 = all) is recomputed with the exact
 * kernel; a judged row whose max |R - R_exact| exceeds tol is replaced by the exact
 * spectrum.  n_fallback (device int32) and max_err (device f32, largest judged
 * error) may be NULL. */
TMM_API tmm_status tmm_surrogate_infer(tmm_surrogate *s, const float *d, int32_t B, float *R, float judge_fraction,
                                       float tol, int32_t *n_fallback, float *max_err, void *stream);
/* Read-only view of layer i (0 .. depth; depth = the head): device pointers to
 * the fp32 master weights W [N][K] (input columns >= Kvalid are zero padding),
 * bias [N], and the gradients dW, db of the last train_step (taken before its
 * Adam update). */
typedef struct {
    int32_t N, K, Kvalid;
    const float *W, *b, *dW, *db;
} tmm_surrogate_layer_view;
TMM_API tmm_status tmm_surrogate_layer(const tmm_surrogate *s, int32_t i, tmm_surrogate_layer_view *out);
/* TMM_OK, or TMM_ERR_TIMEOUT if a tensor-core pipeline wait of this object's last
 * generate / train_step / infer expired (its own flag; synchronises `stream`). */
TMM_API tmm_status tmm_surrogate_status(tmm_surrogate *s, void *stream);
/* Checkpoint: weights, Adam moments and step count (host file). */
TMM_API tmm_status tmm_surrogate_save(tmm_surrogate *s, const char *path);
TMM_API tmm_status tmm_surrogate_load(tmm_surrogate *s, const char *path);

/*
 * Allocation-free variant of the persistent launch (no counterpart in the
 * paper; it serves callers that cannot allocate device memory at call time,
 * such as request paths that must not take cudaMalloc's implicit device
 * synchronisation, or programs whose device memory is owned by another
 * allocator).  Same results as tmm_coh_batched_ex with cfg->persistent = 1
 * and a caller workspace, but the scratch (work counter, error flag, sort
 * buckets, stack order) lives in a 1 MiB array inside the library that every
 * GPU which loads it keeps until exit; nothing is allocated or freed.
 *   cfg      may be NULL; persistent is forced on; max_items_per_block must be 0
 *            (there is no workspace to report a timeout through).
 *   prec     TMM_F64, TMM_F32 or TMM_F32D; TMM_F64X returns TMM_ERR_UNSUPPORTED
 *            (the double-float kernel has no persistent form).
 *   Limit    the problem's persistent workspace (tmm_workspace_size with
 *            persistent = 1: about 4 * (S + 2 * (L_max + 2)) bytes plus
 *            headers) must fit in 1 MiB, i.e. up to ~261,000 stacks for small
 *            L_max; larger problems return TMM_ERR_NOMEM before any launch.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any stream
 *   capture.  The address is kept for the life of the process: do not call
 *   this entry point after cudaDeviceReset of a device it has run on.  Every call shares the one array: calls whose work overlaps on the
 *   GPU (several streams, several host threads) race and must be serialised
 *   by the caller.  Each call zeroes what must start at zero itself.
 */
TMM_API tmm_status tmm_coh_batched_noalloc(const tmm_problem *p, const tmm_launch_cfg *cfg, void *R, void *T,
                                           void *stream);

/*
 * Building block of the learned surrogate, exported for testing: one bf16
 * tensor-core GEMM (tcgen05, TMA-fed) with a fused epilogue.
 *   D[M][N] = sum_k A[M][k] B[N][k];  A, B device bf16, row-major, K a
 *   multiple of 8 and both base addresses 16-byte aligned.
 *   epilogue 0: out f32 [M][N] = D + bias        (bias device [N] or NULL)
 *            1: aux bf16 [M][N] = D + bias; out bf16 = GELU(aux), erf form
 *               z Phi(z) = 0.5 z (1 + erf(z / sqrt 2))
 *            2: out bf16 = D * GELU'(aux)        (aux device bf16 [M][N], read)
 *            3: out f32 = clamp(D + bias, 0, 1)
 * Synchronises `stream` and reports TMM_ERR_TIMEOUT if a pipeline wait of the
 * kernel expired (the kernel then returns without finishing its tile).
 */
TMM_API tmm_status tmm_gemm_bf16(const void *A, const void *B, const float *bias, int32_t M, int32_t N,
                                 int32_t K, int32_t epilogue, void *out, void *aux, void *stream);

/*
 * tmm_gemm_bf16 with epilogue 1 or 2 that also writes the transposed copy
 * outT bf16 [N][ldoT] (outT[n][m] = out[m][n], ldoT >= M; the columns past M
 * are left untouched), as the surrogate's training step does for its weight
 * gradients.  Exported for testing; no paper counterpart.  Other epilogues and
 * a NULL outT return TMM_ERR_INVALID_ARG.
 */
TMM_API tmm_status tmm_gemm_bf16_t(const void *A, const void *B, const float *bias, int32_t M, int32_t N,
                                   int32_t K, int32_t epilogue, void *out, void *aux, void *outT, int32_t ldoT,
                                   void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TMM_GB300_TMM_H */
