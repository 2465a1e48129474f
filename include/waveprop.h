/*
 * waveprop: 3D pseudo-acoustic TTI, isotropic elastic (3D and the x-z
 * plane) and isotropic acoustic wave propagators, their exact adjoints and
 * FWI gradients, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Louboutin et al., "Scaling through abstractions - high-performance
 * vectorial wave simulations for seismic inversion with Devito" (SC20).
 *   - forward operator: model + source wavelet -> receiver traces, with the
 *     source injected (s.inject(u.forward, expr=s*dt**2/m)) and the data
 *     interpolated (d.interpolate(u)): Sec. II-A, Eq. (acou) and the
 *     wave-equation listing;
 *   - TTI system with rotated self-adjoint second derivatives
 *     G_xbarxbar = D_xbar^T D_xbar: Sec. III-A, Eq. (rot);
 *   - elastic velocity-stress system on staggered grids with a damping
 *     factor: Sec. IV, Eq. (elas1) and the elastic listing;
 *   - adjoints ("propagators along with their adjoints", abstract) and the
 *     adjoint-state gradient (zero-lag cross-correlation of forward and
 *     adjoint wavefields), exactness required: Sec. III-A;
 *   - checkpointing of forward wavefields: Sec. III;
 *   - many independent shots (RTM/FWI over experiments): Sec. III-B.
 *
 * Conventions (every entry point):
 *   - Grids are indexed [x][y][z], z fastest, float32.  The PHYSICAL grid has
 *     nx*ny*nz points at spacing h; the library adds nbl absorbing cells on
 *     every face (computational grid (nx+2nbl)(ny+2nbl)(nz+2nbl)) and fills
 *     the layer by edge replication of the model.
 *   - Coordinates are metres, origin at the first physical point, z = depth;
 *     every source/receiver must lie inside the computational grid,
 *     [-nbl h, (n-1+nbl) h] on each axis (PROP_EINVAL otherwise; y = 0 for
 *     PROP_ELASTIC2D, which has no absorbing cells in y).
 *   - Buffers may be host or device pointers (detected per pointer with
 *     cudaPointerGetAttributes).  The caller owns every buffer passed in or
 *     out; the library owns the handle and all device memory it allocates,
 *     and frees it in prop_destroy.
 *   - All work is enqueued on the stream given at prop_create (NULL = the
 *     legacy default stream); every call returns after that work completed.
 *   - Negative return = error.  After PROP_EINVAL the handle stays usable;
 *     after PROP_ECUDA or PROP_ETIMEOUT every later call returns PROP_ESTATE
 *     until prop_destroy.  prop_last_error gives the message.
 *   - One handle per host thread at a time.
 *
 * Measurement hooks (device time per kernel group, launch counts, the FP32
 * peak) and the wait self-test are declared in waveprop_diag.h.
 */
#ifndef WAVEPROP_H
#define WAVEPROP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prop_s prop_t;

enum {
    PROP_OK = 0,
    PROP_EINVAL = -1,     /* bad argument (message says which)             */
    PROP_ENOMEM = -2,     /* device allocation failed (nothing leaked)     */
    PROP_ECUDA = -3,      /* CUDA runtime error, or (WAVEPROP_CHECK=1
                             build) a device bounds check failed; handle
                             unusable                                      */
    PROP_EUNSTABLE = -4,  /* dt violates the CFL bound, or NaN/Inf seen    */
    PROP_ETIMEOUT = -5,   /* a bounded device-side wait gave up            */
    PROP_ESTATE = -6      /* handle unusable after an earlier error,
                             or a call that needs a saved forward run      */
};

/* PROP_ACOUSTIC: the isotropic acoustic equation of Sec. II-A, Eq. (acou),
 * m u_tt - laplace(u) + damp u_t = q, laplace = sum over axes of the centred
 * second derivative of the space order, damped like TTI.
 * PROP_ELASTIC2D: the elastic system in the x-z plane (ny = 1, no absorbing
 * cells on the y faces; source and receiver y = 0), as in the 2D example of
 * Sec. IV-B: fields vx, vz, txx, tzz, txz; explosive source into txx and tzz;
 * receivers record txx + tzz.  Forward and adjoint modelling and state
 * stepping (forward only); no gradient or saved forward run (PROP_EINVAL). */
enum { PROP_TTI = 1, PROP_ELASTIC = 2, PROP_ACOUSTIC = 3, PROP_ELASTIC2D = 4 };

/* Storage of forward wavefields for the gradient (Sec. III: full storage in
 * memory, or checkpointing).  CKPT_* keep the full state every
 * ckpt_interval steps and recompute the segment in FP32 during the adjoint
 * sweep; BF16/FP16 store each checkpoint field with one FP32 scale. */
enum { SNAP_FULL_FP32 = 0, SNAP_CKPT_FP32 = 1, SNAP_CKPT_BF16 = 2, SNAP_CKPT_FP16 = 3 };

typedef struct {
    int kind;            /* PROP_TTI, PROP_ELASTIC, PROP_ACOUSTIC or
                            PROP_ELASTIC2D                                    */
    int nx, ny, nz;      /* physical grid points (>= 1)                       */
    int nbl;             /* absorbing cells added on every face (>= 0; not on
                            the y faces of PROP_ELASTIC2D)                    */
    float h;             /* grid spacing [m] (> 0)                            */
    int space_order;     /* 4, 8, 12 or 16                                    */
    int nt;              /* time samples per trace (>= 2)                     */
    float dt;            /* time step [s]; <= 0 selects dt = 0.4 h / vmax     */
    float vdamp;         /* TTI/acoustic damping reference velocity [m/s];
                            <= 0: the model's max vp sqrt(1+2 eps) (max vp)  */
    int snap_mode;       /* SNAP_* for prop_gradient / prop_backward          */
    int ckpt_interval;   /* steps between checkpoints; 0 = ceil(sqrt(nt))     */
    int check_nan;       /* nonzero: stencil kernels flag NaN/Inf, reported
                            as PROP_EUNSTABLE at the end of the call          */
    int tti_operator;    /* TTI only: 0 = rotated operators of Sec. III-A with
                            composed centred first derivatives; 1 = staggered
                            pair on the diagonal terms: D-_i (P_ii~ D+_i u),
                            P_ii~ the two-node average of the projector's
                            diagonal (P0 = I - n n^T for H0, n n^T for Hz) at
                            the half point, cross terms centred; no
                            checkerboard null vector.  Must be 0 for the other
                            kinds; 1 is not available to
                            prop_forward_noalloc (PROP_EINVAL).               */
} prop_desc;

/* Create a propagator.  model points to the PHYSICAL-grid float32 arrays
 *   TTI:     vp [km/s], epsilon, delta, theta (tilt) [rad], phi (azimuth) [rad]
 *   ELASTIC, ELASTIC2D: vp [km/s], vs [km/s], rho [g/cc]
 *   ACOUSTIC: vp [km/s]
 * (Sec. III-A: 4 Thomsen/angle parameters + velocity; Sec. IV: Lame
 * parameters and density, lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2).
 * The arrays are copied; they may be freed after the call.
 * Errors: PROP_EINVAL for bad sizes, space order, non-positive velocity or
 * density, eps < delta (TTI stability needs eps >= delta), lambda < 0;
 * PROP_EUNSTABLE if dt exceeds the scheme's CFL bound.
 * cuda_stream: a cudaStream_t (NULL = default stream). */
int prop_create(const prop_desc *desc, const float *const *model, void *cuda_stream,
                prop_t **out);

/* Forward modelling (Sec. II-A listing order per step n = 0..nt-1):
 * record d^n from u^n, advance, inject q^n.
 *   wavelet  [nsrc][nt]  source time functions q
 *   src_xyz  [nsrc][3]   source positions
 *   rec_xyz  [nrec][3]   receiver positions
 *   traces   [nrec][nt]  output: TTI records p; ELASTIC records
 *                        txx + tyy + tzz (trace of stress, Sec. IV-B);
 *                        ACOUSTIC records u.
 * TTI injects q into both p and r; ACOUSTIC into u (both with dt^2 / A,
 * A = m (1 + sig dt/2)); ELASTIC injects dt q into txx, tyy, tzz
 * (explosive source).  nsrc, nrec >= 1. */
int prop_forward(prop_t *p, const float *wavelet, const float *src_xyz, int nsrc,
                 const float *rec_xyz, int nrec, float *traces);

/* Adjoint modelling: the exact transpose of prop_forward (as a linear map
 * from wavelets to traces).  traces_in [nrec][nt] -> src_out [nsrc][nt]. */
int prop_adjoint(prop_t *p, const float *traces_in, const float *rec_xyz, int nrec,
                 const float *src_xyz, int nsrc, float *src_out);

/* FWI gradient of J = 1/2 ||F(model) q - d_obs||^2 by the adjoint-state
 * method (zero-lag cross-correlation of forward and adjoint wavefields).
 *   d_obs  [nrec][nt]
 *   grad   TTI, ACOUSTIC: [nx][ny][nz] dJ/dm, m = 1/vp^2 [s^2/m^2] on the
 *          physical grid (layer contributions folded back through the edge
 *          replication);
 *          ELASTIC: [3][nx][ny][nz] dJ/d(lambda [Pa], mu [Pa], b = 1/rho [m^3/kg])
 *   misfit J (may be NULL).
 * Forward wavefields are kept according to desc.snap_mode. */
int prop_gradient(prop_t *p, const float *wavelet, const float *src_xyz, int nsrc,
                  const float *rec_xyz, int nrec, const float *d_obs, float *grad,
                  double *misfit);

/* TTI only: the same gradient also with respect to the anisotropy
 * parameters, from the same forward and adjoint sweeps.  The step depends on
 * epsilon and delta only through the coupling matrix C of Sec. III-A, so
 * with h^n = [H0 p^n; Hz r^n] of the forward field and lam^{n+1} the adjoint
 * field of the same step:
 *   dJ/deps   = sum_n 2 dt^2 lam_p^{n+1} H0 p^n,
 *   dJ/ddelta = sum_n dt^2 (lam_p^{n+1} Hz r^n + lam_r^{n+1} H0 p^n) / sqrt(1 + 2 delta).
 * It depends on the tilt theta and azimuth phi only through the symmetry
 * axis n of Eq. (rot) inside H0 and Hz; with zeta = C lam^{n+1}, g = D p^n,
 * h = D r^n (centred first derivatives at the point) and
 *   V = D zeta_p (n.g) + (n.D zeta_p) g - D zeta_r (n.h) - (n.D zeta_r) h,
 *   dJ/dtheta = sum_n dt^2 dn/dtheta . V,   dJ/dphi = sum_n dt^2 dn/dphi . V
 * (each folded onto the physical grid like dJ/dm).  With tti_operator = 1
 * the diagonal terms use half-point averages of P_ii, so V gains
 *   2 n_i (T0_i - (D_i zeta_p) g_i) - 2 n_i (Tz_i - (D_i zeta_r) h_i),
 * T_i the products (D+_i zeta)(D+_i u) of the half points beside the node
 * (weights 1/2; 1 above the last node, none below the first).
 *   grad  [5][nx][ny][nz]: dJ/dm, dJ/deps, dJ/ddelta, dJ/dtheta, dJ/dphi.
 * Costs per step one more application of H to the stored forward field and
 * the first derivatives of zeta and of the forward field; needs 6 more
 * scratch fields than prop_gradient.
 * Any computational nz with the centred operators (TMA-fed passes when nz +
 * 2 nbl is a multiple of 4, the pipelined passes otherwise).
 * PROP_EINVAL for a non-TTI handle, or for tti_operator = 1 with a
 * computational nz that is not a multiple of 4 (its half-point imaging runs
 * on the TMA-fed passes, which need 16-byte rows). */
int prop_gradient_aniso(prop_t *p, const float *wavelet, const float *src_xyz, int nsrc,
                        const float *rec_xyz, int nrec, const float *d_obs, float *grad,
                        double *misfit);

/* Two-phase form of prop_gradient for automatic differentiation:
 * prop_forward_saved runs prop_forward and keeps the forward wavefields
 * (snap_mode) in the handle; prop_backward then takes the trace gradient
 * resid [nrec][nt] (dJ/dtraces) and returns grad (as prop_gradient, may be
 * NULL) and src_grad [nsrc][nt] = dJ/dwavelet (may be NULL).  prop_backward
 * without a saved forward run returns PROP_ESTATE; it releases the saved
 * wavefields. */
int prop_forward_saved(prop_t *p, const float *wavelet, const float *src_xyz, int nsrc,
                       const float *rec_xyz, int nrec, float *traces);
int prop_backward(prop_t *p, const float *resid, float *grad, float *src_grad);

/* Forward modelling of many independent shots in lockstep (Sec. III-B):
 * shot i computes exactly prop_forward(shots[i], wavelet[i], src_xyz[i],
 * nsrc[i], rec_xyz[i], nrec[i], traces[i]) -- bitwise the same traces.
 * When every shot is TTI with the centred operators (or every shot is
 * elastic), with the same space order and nt, a computational nz that is a
 * multiple of 4 and windows of at most 16 M computational points on
 * average (WAVEPROP_LOCKSTEP=1: any size, =0: never), each time step is
 * one launch of each pass over a table of all the shots' tiles (each shot
 * keeping its own model window, grid and x-extent) beside the shots'
 * injection and receiver sampling; two steps are captured once as a CUDA
 * graph and replayed (WAVEPROP_GRAPHS=0: direct launches).  The work runs
 * on a private stream ordered after the work already queued on each
 * handle's stream; each handle's stream waits for the batch, and the call
 * is synchronous.  Other shot sets (and WAVEPROP_BATCH_LAUNCH=0) run one
 * prop_forward after another.  Arguments as prop_gradient_batch.  Returns
 * PROP_OK or the first error, with the message "shot i: ..." from
 * prop_last_error(NULL). */
int prop_forward_batch(prop_t *const *shots, int nshots, const float *const *wavelet,
                       const float *const *src_xyz, const int *nsrc, const float *const *rec_xyz,
                       const int *nrec, float *const *traces);

/* Gradients of many independent shots (the paper's embarrassingly parallel
 * loop over sources, Sec. III-B: each shot its own model window, geometry
 * and handle).  Shot i computes exactly prop_gradient(shots[i], wavelet[i],
 * src_xyz[i], nsrc[i], rec_xyz[i], nrec[i], d_obs[i], grad[i], &misfit[i])
 * -- bitwise the same result.  Shots are grouped, in order, into waves
 * whose prop_gradient_bytes sum to at most budget_bytes (0: 90 % of the
 * free device memory at the call); the shots of a wave run concurrently,
 * each from its own host thread on a private stream that is ordered after
 * the handle's stream, which in turn waits for the shot.  All handles must
 * be distinct and live on the calling thread's current device; the caller
 * must not use them from another thread during the call.  misfit [nshots]
 * may be NULL.  Returns PROP_OK, or the error of the first failing shot
 * (its message, prefixed "shot i: ", from prop_last_error(NULL); each
 * handle keeps its own message); the other shots still run.  Each shot's
 * work arrays are released after its gradient (prop_trim), so later waves
 * can use that memory; its wavefield state then reads as zero.
 * TTI shots of a wave (centred operators, computational nz a multiple of 4)
 * share their step launches: the k-th step of every such shot runs as one
 * launch of each pass over a table of all the shots' tiles (set
 * WAVEPROP_BATCH_LAUNCH=0 to launch shot by shot).  A wave whose shots are
 * all such TTI shots, or all elastic shots on the TMA-fed passes, with
 * checkpoints (FP32, BF16 or FP16), one space
 * order, nt and checkpoint interval, on windows of at most 16 M
 * computational points on average, runs in lockstep from the calling
 * thread: per step one launch of each pass for every shot, and each full
 * checkpoint segment (the forward steps between two checkpoints; the
 * recomputation and the transposed steps of a segment) replayed from a
 * CUDA graph (WAVEPROP_LOCKSTEP=1: for any window size, =0: never;
 * WAVEPROP_GRAPHS=0: direct launches). */
int prop_gradient_batch(prop_t *const *shots, int nshots, const float *const *wavelet,
                        const float *const *src_xyz, const int *nsrc, const float *const *rec_xyz,
                        const int *nrec, const float *const *d_obs, float *const *grad,
                        double *misfit, size_t budget_bytes);

/* Image stacking over shots (reverse-time migration of many experiments,
 * Sec. III-B): adds weight * image ([nx][ny][nz], the handle's physical
 * grid, e.g. its dJ/dm; host or device) into stack ([sx][sy][sz] =
 * stack_dims, DEVICE memory) with the window's first point at offset
 * (ox, oy, oz), on the handle's stream; returns when done.  The caller
 * serialises calls that target the same stack (a handle's calls are
 * ordered on its stream).  PROP_EINVAL for NULL arguments, a host stack or
 * a window that does not fit. */
int prop_stack_image(prop_t *p, const float *image, float *stack, const int *stack_dims,
                     const int *offset, float weight);

/* Release the handle's work arrays (wavefield state, adjoint state,
 * scratch fields, saved forward run) and keep the model: the next call
 * allocates what it needs again (the state restarts at zero).  A batch of
 * many shots can thus hold all its handles at the size of their models;
 * prop_gradient_batch trims each shot after its gradient.  Synchronises the
 * handle's stream. */
int prop_trim(prop_t *p);

/* Device bytes a prop_gradient call with nrec receivers would allocate on
 * top of what the handle holds (0 for p == NULL). */
size_t prop_gradient_bytes(const prop_t *p, int nrec);

/* The wave plan of prop_gradient_batch: shot i (of n, needing bytes[i]) goes
 * to wave wave_of[i]; waves are filled first-fit in shot order up to budget,
 * a shot above the budget alone.  Returns the number of waves, or PROP_EINVAL
 * for n < 0 or NULL arrays with n > 0.  Host only. */
int prop_plan_waves(const size_t *bytes, int n, size_t budget, int *wave_of);

/* Wavefield state access (computational grid, float32 [NX][NY][NZ] each):
 *   TTI:     fields[0..3] = p^n, r^n, p^{n-1}, r^{n-1}
 *   ACOUSTIC: fields[0..1] = u^n, u^{n-1}
 *   ELASTIC2D: fields[0..4] = vx vz txx tzz txz (prop_step: forward only)
 *   ELASTIC: fields[0..8] = vx vy vz txx tyy tzz txy txz tyz
 * prop_step advances nsteps steps without sources or receivers (adjoint != 0:
 * transposed step, state holds the adjoint fields in the same order).  From
 * nsteps >= 4 on, pairs of steps replay a CUDA graph captured once per handle,
 * direction and state buffers (results bitwise those of direct launches);
 * environment WAVEPROP_GRAPHS=0 launches every step directly, =1 makes a
 * failed capture an error (PROP_EINVAL) instead of a silent direct run. */
int prop_grid_dims(const prop_t *p, int *dims /* [3] = NX, NY, NZ */, int *nfields);
int prop_set_state(prop_t *p, const float *const *fields);
int prop_get_state(prop_t *p, float *const *fields);
int prop_step(prop_t *p, int nsteps, int adjoint);

/* Time step actually used (after the CFL rule), in seconds. */
float prop_dt(const prop_t *p);

/* Tile shape of the x-streaming stencil kernels: a CTA updates a tile of
 * 32 (z) x prop_tile_rows (y) columns over prop_tile_planes planes of x.
 * prop_create picks both by timing a few steps of the zero state for a set
 * of candidates: heights 8, 16 and 32 rows for the elastic and centred TTI
 * passes on the TMA path (16 for the others), x-extents from NX down to 8
 * planes.  The choice is cached per kind, space order, grid and kernel
 * family for the process; environment WAVEPROP_AUTOTUNE_CACHE=<file> keeps
 * the cache across processes, WAVEPROP_AUTOTUNE=0 skips the timing and keeps
 * an occupancy heuristic at 16 rows, WAVEPROP_TILE_Y=8|16|32 fixes the
 * height.  Results are bitwise independent of the choice.  Both return 0
 * for p == NULL. */
int prop_tile_planes(const prop_t *p);
int prop_tile_rows(const prop_t *p);

/* Forward modelling that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc, e.g. an
 * application whose own allocator has already reserved the GPU's memory, or
 * a latency-bound service that forbids device allocation after start-up
 * (cudaMalloc/cudaFree can synchronize the device).  It computes exactly what
 * prop_create(desc, model, cuda_stream) + prop_forward(...) + prop_destroy
 * would, with the same arguments, conventions and error codes, but every
 * device buffer it needs lives in one static device array of 48 MiB that the
 * library keeps on each GPU where it is used, from the first call there until
 * the process exits.  Problems that do not fit (TTI needs about 68 bytes per
 * computational grid point, elastic about 48, plus the wavelet, traces and
 * point tables) are rejected with PROP_EINVAL and a message giving the size.
 * The first call on a device looks up the array's address; make that first
 * call before starting any stream capture on that device.  All calls share
 * the array (contents are cleared as needed on each call): calls that overlap
 * on the GPU -- concurrent streams or host threads -- race and must be
 * serialised by the caller.  Errors are reported through prop_last_error(NULL). */
int prop_forward_noalloc(const prop_desc *desc, const float *const *model, const float *wavelet,
                         const float *src_xyz, int nsrc, const float *rec_xyz, int nrec,
                         float *traces, void *cuda_stream);

void prop_destroy(prop_t *p);                 /* NULL-safe */

/* Message of the last error on this handle; with p == NULL, the last
 * error of the calling thread (e.g. a failed prop_create). */
const char *prop_last_error(const prop_t *p);

#ifdef __cplusplus
}
#endif
#endif /* WAVEPROP_H */
