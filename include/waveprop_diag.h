/*
 * waveprop measurement and self-test hooks.  None of these calls changes
 * what the propagators compute; they serve roofline accounting (device time
 * of the stencil kernels, launch counts, the FP32 peak that bounds the
 * arithmetic side of the stencil roofline) and the tests of the failure
 * paths.  The conventions of waveprop.h hold: negative return = error,
 * prop_last_error gives the message, one handle per host thread at a time.
 */
#ifndef WAVEPROP_DIAG_H
#define WAVEPROP_DIAG_H

#include "waveprop.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel groups of prop_kernel_stats.  Each group is one time step of a
 * propagator (all its stencil passes), bracketed by two CUDA events on the
 * handle's stream:
 *   PROP_K_TTI_FWD      TTI step (rotation and update passes)
 *   PROP_K_TTI_ADJ      TTI transposed step, with or without imaging
 *   PROP_K_EL_FWD       elastic step (velocity and stress passes)
 *   PROP_K_EL_ADJ       elastic transposed step on the direct-load kernels
 *   PROP_K_EL_ADJ_GRAD  elastic transposed step with imaging (Sec. III-A
 *                       gradient w.r.t. lambda, mu, b)
 *   PROP_K_EL_ADJ_U     elastic step with dt negated (the transposed step in
 *                       the transformed variables of the TMA-fed path)
 *   PROP_K_AC_STEP      acoustic step
 *   PROP_K_AC_IMG       acoustic transposed step with imaging
 * Source injection, receiver interpolation and the pointwise kernels of a
 * step are not inside the brackets. */
enum {
    PROP_K_TTI_FWD = 0,
    PROP_K_TTI_ADJ = 1,
    PROP_K_EL_FWD = 2,
    PROP_K_EL_ADJ = 3,
    PROP_K_EL_ADJ_GRAD = 4,
    PROP_K_EL_ADJ_U = 5,
    PROP_K_AC_STEP = 6,
    PROP_K_AC_IMG = 7,
    PROP_K_GROUPS = 8
};

/* on != 0 starts recording the device time of every step of the handle
 * (two CUDA event records per step, no synchronisation inside a sweep; the
 * events are read at the end of each call and every 256 steps), on == 0
 * stops it.  Either way the pending events are read first and every
 * counter is then set to zero.  PROP_EINVAL for p == NULL. */
int prop_profile(prop_t *p, int on);

/* Device time [ms] summed over the recorded steps of group id, and the
 * number of those steps, since the last prop_profile.  Complete after every
 * call on the handle has returned; zero while profiling is off.  Either
 * output may be NULL.  PROP_EINVAL for p == NULL or id outside
 * [0, PROP_K_GROUPS). */
int prop_kernel_stats(const prop_t *p, int id, double *ms, long long *steps);

/* The same sums over every group (*steps: recorded steps).  PROP_EINVAL
 * for p == NULL. */
int prop_kernel_time(const prop_t *p, double *ms, long long *steps);

/* Kernel launches the library made for the handle during its most recent
 * call (every kernel: stencil passes, injection, interpolation, pointwise,
 * encode/decode of snapshots; a replayed CUDA graph counts the launches it
 * holds, and a launch that advances several shots of a batch counts once
 * for each of them; prop_trim leaves the count as it is, so after a batch
 * call it is the count of that call).  0 for p == NULL. */
long long prop_last_launches(const prop_t *p);

/* Steps of the most recent prop_gradient_batch call made by the calling
 * host thread: *shared = rounds in which one launch of each pass advanced
 * several shots (rendezvous rounds and lockstep steps), *alone = rendezvous
 * rounds whose steps had to be launched shot by shot.  Either output may be
 * NULL.  Always PROP_OK. */
int prop_batch_stats(long long *shared, long long *alone);

/* Measured FP32 throughput of the current device [TFLOP/s]: chains of
 * fused multiply-adds (2 FLOP each) on every SM, best of three timed
 * launches after a warm-up, on the legacy default stream; allocates and
 * frees a few KB of device memory and synchronises the device.
 * PROP_EINVAL for tflops == NULL, PROP_ENOMEM, PROP_ECUDA. */
int prop_fp32_peak(double *tflops);

/* Failure-path self-test of the bounded device-side waits: one kernel waits
 * on a shared-memory mbarrier that nothing completes, gives up after
 * `seconds` (clamped to [0, 2]), records the expiry in the handle's device
 * flag word and returns; the call then returns PROP_ETIMEOUT exactly as an
 * expired wait of a TMA pipeline does, the handle reports PROP_ESTATE from
 * then on, and the CUDA context stays usable.  PROP_EINVAL for p == NULL, PROP_ESTATE
 * for a handle already unusable. */
int prop_selftest_wait(prop_t *p, float seconds);

#ifdef __cplusplus
}
#endif
#endif /* WAVEPROP_DIAG_H */
