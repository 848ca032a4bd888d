/*
 * tpflbm — GB300 (sm_103a) library for the phase-field thermocapillary lattice
 * Boltzmann method of Wang, He & Wang, "Phase-field-based lattice Boltzmann model
 * for simulating thermocapillary flows" (arXiv 2306.11320).
 *
 * One lattice of nx x ny nodes (D2Q9, dx = dt = 1, Sec. 4) carries three sets of
 * populations: f (conservative Allen-Cahn LBE, Eq. 14), g (pressure-based
 * Navier-Stokes LBE, Sec. 3.1) and h (the heat-capacitance weighted thermal LBE,
 * Eq. 28).  tpflbm_step advances all three by one time step per call of the
 * fused step kernel: moments, isotropic stencils, closures (Eq. 45), interfacial
 * force with the Marangoni stress (Eq. 11), BGK collisions, streaming and the
 * wall / inlet / outflow rules of Sec. 4.
 *
 * Conventions for every call:
 *   - Return value 0 (TPF_OK) on success, a negative TPF_ERR_* code otherwise; the
 *     message of the last failure on a handle is tpflbm_last_error(handle).  No C++
 *     exception crosses this interface.
 *   - Fields are float32, row-major [ny][nx], y = 0 the bottom fluid row; walls sit
 *     halfway, at y = -1/2 and y = ny - 1/2; the inlet at x = -1/2, the outflow
 *     plane at x = nx - 1/2.  Populations are [9][ny][nx] per LBE in the D2Q9 order
 *     of Eq. 43: rest, (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
 *   - A field pointer may point to host memory or to device memory of the
 *     handle's device; the library finds out which.  Caller-owned buffers stay
 *     caller-owned; the library copies what it needs before returning.
 *   - Work is ordered on the handle's CUDA stream (tpflbm_set_stream; default:
 *     the legacy default stream).  Calls that return data to the caller
 *     synchronise that stream before returning.
 */
#ifndef TPFLBM_H
#define TPFLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPF_OK 0
#define TPF_ERR_INVALID_ARG (-1)
#define TPF_ERR_OOM (-2)
#define TPF_ERR_CUDA (-3)
#define TPF_ERR_NONFINITE (-4)
#define TPF_ERR_TIMEOUT (-5)
#define TPF_ERR_UNSUPPORTED (-6)

#define TPF_STORAGE_FP32 0 /* populations stored as float32 */
#define TPF_STORAGE_FP16 1 /* populations stored as scaled float16 deviations */

typedef struct tpflbm *tpflbm_t;

/* Physical parameters in lattice units (Sec. 2-4 of the paper).
 *   rho, mu, lambda, cp (_l light phase phi = -1, _h heavy phase phi = +1):
 *       interpolated linearly in phi, Eq. 45 (rho also Eq. 8); tau_g from
 *       mu = rho cs2 (tau_g - 1/2), tau_h from lambda = cs2 (tau_h - 1/2).
 *   W, M_phi: interface width and mobility, M_phi = cs2 (tau_phi - 1/2) (Sec. 3.1).
 *   sigma_law 0: sigma = sigma_ref + sigma_T (T - T_ref) (Eq. 12);
 *   sigma_law 1: sigma = sigma_TT (T - T_ref)^2 / 2 + sigma_ref (Eq. 63).
 *   Gx, Gy: body-force density G of Eq. 7.
 *   bc_x 0: periodic in x; 1: velocity inlet u_x(y) = 6 u_ave y (H - y) / H^2 with
 *       phi = phi_in and T = T_in at x = -1/2, stress-free outflow (p = p_out,
 *       zero-gradient phi and T) at x = nx - 1/2 (Sec. 4.3).
 *   bc_y 0: halfway no-slip walls with Dirichlet temperature
 *       T_bottom(x) = T_bot + T_bot_amp cos(2 pi T_bot_k x / nx) + T_bot_slope x,
 *       T_top(x) = T_top + T_top_slope x (Sec. 4.1-4.3); 1: periodic in y.
 *   collision: 0 BGK for every LBE (Sec. 3); 1 two relaxation times for the NS and
 *       thermal LBEs (the stability extension the paper points to in Sec. 3): with
 *       X^{+/-} = (X_i +/- X_opp(i))/2 the even and odd parts relax at 1/tau+ and
 *       1/tau-, (tau+ - 1/2)(tau- - 1/2) = trt_lambda (> 0), tau+ = tau_g for g
 *       (viscosity), tau- = tau_h for h (conductivity); the NS source splits with
 *       factors 1 - 1/(2 tau+/-).  trt_lambda = 3/16 makes halfway bounce-back walls
 *       exact for Poiseuille flow; (tau - 1/2)^2 gives BGK back.
 *   normal_law: interface normal n in the Allen-Cahn source R_i (Eq. 14): 0 from the
 *       isotropic stencil gradient of phi; 1 recovered locally from the populations
 *       (Sec. 3): n = -J / |J| with J = sum_i c_i (f_i - f_i^eq) + d_t(phi u) / 2.
 *   storage: TPF_STORAGE_FP32 or TPF_STORAGE_FP16.  With FP16 a population q_i of
 *       LBE k is stored in float16 as s_k (q_i - r_i), its deviation from a
 *       reference that the node which wrote it (the node it streamed from; for a
 *       population reflected at a boundary the node itself; for f, h entering through
 *       the outflow the last-column node that copied it) leaves for it: the rest
 *       equilibrium plus the first-order term of what that node emitted,
 *       r_i = w_i (phi + c_i . J_f / cs2) for f, w_i (T + c_i . J_h / cs2) for h,
 *       wg_i p / cs2 + w_i c_i . J_g / cs2 for g (wg_0 = w_0 - 1, wg_i = w_i), with J
 *       the first moment of the post-collision populations.  Each node keeps one
 *       8-byte record per LBE for this: the zeroth moment (phi, p / cs2, T) in float32
 *       and J / cs2 as two halves.
 *       s_k are powers of two, fp16_scale_f/g/h (0 selects the defaults 1024, 1024,
 *       64).  All arithmetic stays float32.
 */
typedef struct tpflbm_params {
    double rho_l, rho_h, mu_l, mu_h, lambda_l, lambda_h, cp_l, cp_h;
    double W, M_phi;
    double sigma_ref, sigma_T, sigma_TT, T_ref;
    double Gx, Gy;
    double u_ave, phi_in, T_in, p_out;
    double T_bot, T_bot_amp, T_bot_k, T_bot_slope, T_top, T_top_slope;
    double fp16_scale_f, fp16_scale_g, fp16_scale_h;
    double trt_lambda;
    int sigma_law, bc_x, bc_y, storage, normal_law, collision;
} tpflbm_params;

/* Device bytes tpflbm_create_in needs for an nx x ny lattice with these
 * parameters (both population buffers, (phi u) of the previous step, field and
 * reduction scratch).  Returns 0 for invalid sizes. */
size_t tpflbm_workspace_bytes(int nx, int ny, const tpflbm_params *p);

/* Create a lattice; the library allocates its device memory (cudaMalloc) on the
 * current device and frees it in tpflbm_destroy.  nx, ny >= 3; relaxation times
 * must exceed 1/2.  *out receives the handle. */
int tpflbm_create(int nx, int ny, const tpflbm_params *p, tpflbm_t *out);

/* Same, in caller-owned device memory `workspace` of at least
 * tpflbm_workspace_bytes(nx, ny, p) bytes, 256-byte aligned, on the current
 * device; the caller keeps it alive until tpflbm_destroy and frees it after. */
int tpflbm_create_in(int nx, int ny, const tpflbm_params *p, void *workspace, size_t bytes,
                     tpflbm_t *out);

/* Order all later work of the handle on `stream` (a cudaStream_t; NULL = legacy
 * default stream). */
int tpflbm_set_stream(tpflbm_t h, void *stream);

/* Initial populations from macroscopic fields (the paper gives none):
 * f = f^eq(phi, u), g = g^eq(p, rho(phi), u), h = w_i T (Sec. 3), and the previous
 * (phi u) = phi u.  Each pointer is a [ny][nx] float32 field; NULL means zero
 * (for phi: +1).  Resets the step counter. */
int tpflbm_init(tpflbm_t h, const float *phi, const float *ux, const float *uy, const float *p,
                const float *T);

/* Same fields, with half of forcing sources taken off the equilibria: with bit 0 of
 * `which`, f_i = f_i^eq - R_i / 2 (R_i: the interface term of the Allen-Cahn source,
 * Eq. 14, with d_t(phi u) = 0); with bit 1, g_i = g_i^eq - G_i / 2 (G_i: the NS forcing
 * of Sec. 3.1 with the interfacial force of Eq. 11 at the given phi, T and u).  The
 * step adds its sources as (1 - 1/(2 tau)) S, so with which = 3 these populations
 * decode to the given u and p exactly.  A lattice started near its steady state (a
 * warm start) then skips part of the transient that equilibrium populations excite;
 * which = 1, 2 or 3, anything else is TPF_ERR_INVALID_ARG.  The paper states no
 * initialisation; tpflbm_init stays the plain equilibrium. */
int tpflbm_init_forced(tpflbm_t h, const float *phi, const float *ux, const float *uy, const float *p,
                       const float *T, int which);

/* Advance nsteps >= 0 time steps (one fused step-kernel launch each), enqueued
 * on the handle's stream; returns after enqueueing. */
int tpflbm_step(tpflbm_t h, long long nsteps);

/* Wait for the steps enqueued so far and report whether they completed: TPF_OK, or
 * TPF_ERR_TIMEOUT when a step kernel gave up waiting for its shared-memory copies (a
 * 4-byte device flag read back on the handle's stream), or TPF_ERR_CUDA.  Synchronises
 * the stream. */
int tpflbm_status(tpflbm_t h);

/* The same report without waiting: enqueue a copy of the step kernels' 4-byte error
 * flag into *flag (host memory the caller owns; page-locked for the copy to be
 * asynchronous), ordered after the steps enqueued so far, and return.  copy_stream
 * (cudaStream_t) NULL or the handle's stream: the copy is enqueued on the handle's
 * stream, and later steps queue behind it.  Another stream: the copy is enqueued there
 * behind an event recorded on the handle's stream, and later steps do not wait for it
 * (the flag may then also include a failure of a step enqueued after the call).  Once
 * the copy's stream has passed it (an event recorded there after this call, or any
 * later synchronisation), *flag is 0 if every step enqueued before the call completed
 * and nonzero if a step kernel gave up waiting for its copies.  Lets a caller read
 * each step's outcome while the next steps run.  TPF_OK, or TPF_ERR_CUDA if the copy
 * cannot be enqueued. */
int tpflbm_status_async(tpflbm_t h, int *flag, void *copy_stream);

/* Macroscopic fields of the current state, as the next step computes them:
 * phi = sum f_i, T = sum h_i, u from rho u = sum c_i g_i + (Fs + G)/2 and p from the
 * pressure moment of Sec. 3.1.  Each output is a caller-owned [ny][nx] float32
 * buffer (host or device) or NULL to skip.  Synchronises the stream. */
int tpflbm_get_fields(tpflbm_t h, float *phi, float *ux, float *uy, float *p, float *T);

/* Raw state as float32: f, g, h each [9][ny][nx] (decoded from FP16 storage when
 * used), phiu [2][ny][nx] = (phi u) of the previous step.  NULL skips an array.
 * Synchronises the stream. */
int tpflbm_get_state(tpflbm_t h, float *f, float *g, float *hh, float *phiu);

/* Overwrite the state (same layouts; encoded to FP16 when that storage is used).
 * All four pointers are required. */
int tpflbm_set_state(tpflbm_t h, const float *f, const float *g, const float *hh, const float *phiu);

/* FP64 reductions of the current state (accumulated in double on the device):
 * out[0] sum phi, out[1] sum rho c_p T, out[2] sum T, out[3] U_r numerator
 * sum_{phi<0} phi u_y, out[4] U_r denominator sum_{phi<0} phi, out[5] sum_{phi<0} phi u_x,
 * out[6] sum_{phi<0} phi x, out[7] number of non-finite phi, u or T values.
 * U_r = out[3] / out[4] is the migration velocity of Sec. 4.2.  Synchronises. */
int tpflbm_diagnostics(tpflbm_t h, double out[8]);

/* Same eight reductions as tpflbm_diagnostics, for a state held in caller memory,
 * allocating no device memory at all.  (The paper has no counterpart.  It serves
 * callers that must not call cudaMalloc: code that runs inside a memory pool's or an
 * allocator's own callback, where allocating would re-enter the allocator, and hosts
 * that hand a library only fixed buffers they own and account for.)
 *   pop   device pointer, 27 population planes (f 0-8, g 9-17, h 18-26) of `plane`
 *         elements each, [ny][nx] inside a plane; float32, or float16 encoded as in
 *         tpflbm_params.storage when p->storage is TPF_STORAGE_FP16.
 *   plane elements per plane, >= nx * ny (the buffers must hold 27, 3 and 2 planes).
 *   ref   FP16 storage only: the reference records of the previous step, three
 *         planes (f, g, h) of `plane` 8-byte records (float32 zeroth moment, then
 *         two halves, see tpflbm_params.storage); NULL for FP32.
 *   phiu  device pointer, 2 float planes of `plane` elements ((phi u) of the
 *         previous step).
 *   out   8 doubles, host or device memory; same meaning as tpflbm_diagnostics.
 *   stream cudaStream_t (NULL = legacy default stream); the call synchronises it.
 * tpflbm_state_buffers gives these pointers for a handle's own state.
 * The kernel's scratch (per-block partial sums) is a fixed array of 1024 x 8 + 8
 * doubles (65,600 bytes) compiled into the library; every GPU that loads the
 * library holds it until the process exits.  Any lattice the library accepts
 * (nx, ny >= 3, nx * ny <= 2^30) fits, because the kernel walks the lattice with
 * at most 1024 blocks; larger sizes and invalid arguments return
 * TPF_ERR_INVALID_ARG (message in tpflbm_last_error(NULL)).  Each call looks up the
 * array's address in the current context (cudaGetSymbolAddress, no allocation); on
 * the first call on a device that lookup may also load the library's device code
 * there, so make that first call before any stream capture.  All calls share the
 * array and each call overwrites every entry it reads, so nothing needs clearing;
 * calls whose work overlaps on the GPU (for example on two streams) race on it and
 * must be serialised by the caller. */
int tpflbm_diagnostics_static(int nx, int ny, const tpflbm_params *p, const void *pop, long long plane,
                              const void *ref, const float *phiu, double out[8], void *stream);

/* Device pointers of the handle's current state (time tpflbm_time(h)), as
 * tpflbm_diagnostics_static takes them: *pop the 27 population planes, *ref the three
 * FP16 reference-record planes (NULL with FP32 storage), *phiu the two (phi u) planes,
 * *plane the elements per plane (>= nx * ny, padded).  Any output pointer may be NULL.
 * The pointers stay owned by the handle and change with every step (the two
 * population buffers alternate); read them after the stream has finished the steps. */
int tpflbm_state_buffers(tpflbm_t h, void **pop, void **ref, void **phiu, long long *plane);

/* Per-bubble migration velocity and position of Sec. 4.3 (the paper's u_b,alpha and
 * x_b,alpha, after Eq. 63): the bubbles are the connected regions of phi < 0 of the
 * current state (4-neighbour connectivity, wrapping along periodic axes), labelled on
 * the device; for each, FP64 sums over its nodes give
 *   out[6k + 0] number of nodes,      out[6k + 1] sum phi (negative),
 *   out[6k + 2] u_b = sum phi u_x / sum phi,   out[6k + 3] v_b = sum phi u_y / sum phi,
 *   out[6k + 4] x_b = sum phi x / sum phi,     out[6k + 5] y_b = sum phi y / sum phi,
 * with (x, y) node coordinates (node (x, y) at x, y; along a periodic axis each node is
 * taken at its image nearest to the region's first node, so a bubble that straddles the
 * seam keeps one centroid, reported in [0, nx) or [0, ny)).  Bubbles are ordered by x_b
 * (then y_b); *count receives their number and the first min(*count, max_bubbles) are
 * written to out (6 doubles each; out may be NULL when max_bubbles is 0).  At most 32
 * separate regions are supported (TPF_ERR_UNSUPPORTED beyond).  Uses the lattice's
 * staging and reduction memory (not its state) and synchronises its stream. */
int tpflbm_bubbles(tpflbm_t h, int max_bubbles, double *out, int *count);

/* Steady-state residual (the paper states no convergence criterion; this is the one
 * the warm-start comparison uses).  With u, T the current fields and u', T' those of
 * the previous call, K steps earlier, and N = nx * ny:
 *   out[0] = ||u - u'||_2 / (K ||u||_2),  out[1] = ||T - T'||_2 / (K dT sqrt(N)),
 *   out[2] = K,
 * sums accumulated in FP64 on the device.  The call then keeps the current fields for
 * the next call.  After tpflbm_init the first call has nothing to compare with and
 * returns out[0] = out[1] = +inf, out[2] = 0.  dT > 0 is the temperature scale (e.g.
 * the wall temperature difference).  Synchronises the stream. */
int tpflbm_residual(tpflbm_t h, double dT, double out[3]);

/* Mass-preserving projection of a predicted phase field (the warm start's output;
 * the paper has no warm start).  phi_pred and phi_out are device [ny][nx] float
 * arrays of this lattice's size (they may be the same array).  With the equilibrium
 * profile phi = tanh(d / (sqrt(2) W)) (Sec. 2), the predicted signed distance of each
 * node, a = d / (sqrt(2) W), is taken
 *   mode TPF_PROJECT_ATANH:   as atanh(phi_pred) (phi_pred clipped to |phi| <= 1 - 1e-7);
 *   mode TPF_PROJECT_CONTOUR: as (y_c(x) - y) / (sqrt(2) W), y_c(x) the lowest height
 *       where phi_pred changes sign from positive to non-positive going up column x
 *       (linear interpolation; heavy fluid below, an interface that is a graph over
 *       x, as in the layered channel of Sec. 4.1; a column without a sign change
 *       takes its node of least |phi_pred|).
 * The call finds the uniform offset s for which sum_n tanh(a_n + s) equals target_sum
 * (Newton's method on FP64 device sums, to 1e-12 per node) and writes
 * phi_out = tanh(a + s) in float32.  *achieved (may be NULL) receives the FP64 sum
 * before rounding.  Needs |target_sum| < nx * ny and a field with an interface;
 * uses the lattice's staging memory (not its state) and synchronises its stream. */
#define TPF_PROJECT_ATANH 0
#define TPF_PROJECT_CONTOUR 1
int tpflbm_project_phi(tpflbm_t h, const float *phi_pred, double target_sum, int mode, float *phi_out,
                       double *achieved);

/* Self-check of the step kernels' bounded waits (their failure path, without a GPU
 * fault): one block of 256 threads waits, with the same bounded wait the TMA-staged
 * kernels use (at most `polls` polls here, about 2^22 there), on an mbarrier that
 * nothing completes, then votes and raises a device flag as a step kernel raises its
 * error flag.  *gave_up receives 1 when the wait ran out, the expected outcome, and 0
 * otherwise.  No copy is ever in flight, so the context stays usable.  Runs on the
 * default stream and synchronises it.  Errors: INVALID_ARG (polls < 1 or gave_up
 * NULL), CUDA; the message is in tpflbm_last_error(NULL). */
int tpflbm_check_bounded_wait(int polls, int *gave_up);

/* Number of time steps taken since tpflbm_init. */
long long tpflbm_time(tpflbm_t h);

/* Release the handle and the device memory the library allocated.  NULL-safe. */
void tpflbm_destroy(tpflbm_t h);

/* Message of the last failure on h (or of the last failed create when h is NULL). */
const char *tpflbm_last_error(tpflbm_t h);

/* ------------------------------------------------------------------ ensembles
 * A batch advances n independent lattices (sizes, parameters and boundary kinds may
 * all differ; storage must be the same) together: one persistent launch per time
 * step walks a list of (lattice, tile) pairs and runs the same per-tile step as a
 * single lattice; pairs of steps are replayed from a CUDA graph.  The variant is one
 * of a few compiled ones (tpflbm_batch_variants), chosen by tpflbm_batch_tune or set
 * directly: the general tile path with one of four tile shapes, or (the last
 * variant) 32 x 8 tiles staged by TMA from each lattice's own tensor maps wherever the
 * single-lattice kernel would stage them, the rest through the general path.  If a
 * TMA-staged tile's copies time out, the lattice's next synchronising read-back call
 * reports TPF_ERR_TIMEOUT.  The library allocates every lattice's memory. */
typedef struct tpflbm_batch *tpflbm_batch_t;

/* nx[k], ny[k] (3 <= both < 65536) and params[k] of lattice k = 0..n-1.  The batch
 * works on its own non-blocking stream until tpflbm_batch_set_stream. */
int tpflbm_batch_create(int n, const int *nx, const int *ny, const tpflbm_params *params,
                        tpflbm_batch_t *out);
/* Order the batch's work on `stream` (a non-default cudaStream_t: graphs are captured on it). */
int tpflbm_batch_set_stream(tpflbm_batch_t b, void *stream);
/* Number of lattices. */
int tpflbm_batch_size(tpflbm_batch_t b);
/* The handle of lattice k (owned by the batch; valid until tpflbm_batch_destroy), for
 * the single-lattice read-back calls (tpflbm_get_state, tpflbm_diagnostics, ...). */
int tpflbm_batch_lattice(tpflbm_batch_t b, int k, tpflbm_t *out);
/* tpflbm_init of lattice k (same field conventions). */
int tpflbm_batch_init(tpflbm_batch_t b, int k, const float *phi, const float *ux, const float *uy,
                      const float *p, const float *T);
/* Advance every lattice by nsteps >= 0 time steps; returns after enqueueing. */
int tpflbm_batch_step(tpflbm_batch_t b, long long nsteps);
/* tpflbm_get_fields of lattice k. */
int tpflbm_batch_get_fields(tpflbm_batch_t b, int k, float *phi, float *ux, float *uy, float *p, float *T);
/* tpflbm_diagnostics of every lattice: out[8 k + j], j as in tpflbm_diagnostics. */
int tpflbm_batch_diagnostics(tpflbm_batch_t b, double *out);
/* tpflbm_residual of every lattice: dT[k] the temperature scale of lattice k, out
 * 3 doubles per lattice (n x 3).  Synchronises the batch's stream. */
int tpflbm_batch_residual(tpflbm_batch_t b, const double *dT, double *out);

/* The compiled variants: *count of them, variant v has bx[v] x by[v] node tiles (arrays
 * of at least *count entries, or NULL).  Variant *count - 1 is the TMA-staged one. */
int tpflbm_batch_variants(int *count, int *bx, int *by);
/* Use variant v for the following steps. */
int tpflbm_batch_set_variant(tpflbm_batch_t b, int v);
/* Time every variant over `steps` (>= 2, rounded down to even) steps of the current
 * state and keep the fastest; ms_per_step[v] (or NULL) receives each variant's time
 * per step, *best (or NULL) the chosen one.  The batch advances by
 * count x (steps + 2) steps. */
int tpflbm_batch_tune(tpflbm_batch_t b, int steps, double *ms_per_step, int *best);
/* Steps taken since creation. */
long long tpflbm_batch_time(tpflbm_batch_t b);
/* Release the batch and every lattice in it.  NULL-safe. */
void tpflbm_batch_destroy(tpflbm_batch_t b);
/* Message of the last failure on b (or of the last failed create when b is NULL). */
const char *tpflbm_batch_last_error(tpflbm_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* TPFLBM_H */
