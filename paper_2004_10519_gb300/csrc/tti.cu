// TTI propagator kernels (Sec. III-A).
//
// The rotated operators are applied in their single-axis form: with the
// symmetry axis n = (sin th cos ph, sin th sin ph, cos th) and an orthonormal
// rotated frame (x-bar of Eq. (rot), y-bar, n), G_xbxb + G_ybyb + G_nn =
// sum_i D_i^T D_i pointwise, so with D^T = -D (zero extension)
//     H0 u = -(G_xbxb + G_ybyb) u = sum_i D_i ( D_i u - n_i (n . D u) )
//     Hz u = -G_nn u              = sum_i D_i ( n_i (n . D u) ).
// A step is two passes: (1) the gradient and its rotation into the six
// intermediates e_i = D_i p - n_i (n.Dp), f_i = n_i (n.Dr); (2) the
// divergence H0 p = sum_i D_i e_i, Hz r = sum_i D_i f_i, the coupling
//     L = C [H0 p; Hz r],  C = [[1+2eps, sqrt(1+2delta)], [sqrt(1+2delta), 1]],
// and the damped leapfrog  A u^{n+1} = dt^2 L u^n + 2 m u^n - B u^{n-1},
// A = m(1 + sig dt/2), B = m(1 - sig dt/2).
// The adjoint step is the transpose: C is applied BEFORE the stencil
// (L^T = H C); pass (1) forms zeta = C lam while loading.
//
// The passes themselves live in stencil_tma.cu (TMA-fed, NZ a multiple of
// 4) and tti_fast.cu (pipelined loads, any NZ); this file dispatches a step
// and sizes the x-chunks of the streaming kernels.
#include "common.cuh"

#include <algorithm>

int tti_launch_step(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                    float *grad)
{
    if (P->rdv && tti_batchable(P)) return rdv_tti_step(P, S, adjoint, img_p, img_r, grad);
    if (P->d.tti_operator == 1) return tti_sp_launch(P, S, adjoint, img_p, img_r, grad);
    return tma_usable(P) ? tti_launch_tma(P, S, adjoint, img_p, img_r, grad)
                         : tti_launch_fast(P, S, adjoint, img_p, img_r, grad);
}

// x-chunk length (planes per CTA): enough CTAs for several waves of 2 CTAs
// per SM, rounded so that the CTA count is close to a whole number of waves
// (the autotuner in runtime.cu starts from this value)
int stencil_xchunk(const GridDev &g, int sms)
{
    constexpr int TZ = 32, TY = 16;
    const long long tiles = (long long)((g.NZ + TZ - 1) / TZ) * ((g.NY + TY - 1) / TY);
    const long long slots = 2LL * sms;
    long long chunks = std::max(1LL, (5 * slots + tiles - 1) / tiles);
    long long best = chunks, bestw = 1 << 30;
    for (long long c = std::max(1LL, chunks - 3); c <= chunks + 3; c++) {
        long long ctas = tiles * c, rem = ctas % slots;
        long long waste = rem ? slots - rem : 0;
        if (waste < bestw) { bestw = waste; best = c; }
    }
    int xc = (int)((g.NX + best - 1) / best);
    return std::max(xc, std::min(g.NX, 8));
}
