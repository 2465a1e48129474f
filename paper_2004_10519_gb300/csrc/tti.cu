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
// (L^T = H C), so a pointwise pass forms zeta = C lam first.
#include "common.cuh"

namespace {

constexpr int TZ = 32, TY = 8;

template <int M>
__global__ void __launch_bounds__(TZ *TY)
tti_rot_kernel(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
               const float *__restrict__ th, const float *__restrict__ ph,
               float *__restrict__ ex, float *__restrict__ ey, float *__restrict__ ez,
               float *__restrict__ fx, float *__restrict__ fy, float *__restrict__ fz)
{
    const int z = blockIdx.x * TZ + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int x = blockIdx.z;
    if (z >= g.NZ || y >= g.NY) return;
    const long long q = gidx(g, x, y, z);
    float gp[3] = {0.f, 0.f, 0.f}, gr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const float c = w.c[k - 1];
        gp[0] += c * (ldz(p, g, x + k, y, z) - ldz(p, g, x - k, y, z));
        gp[1] += c * (ldz(p, g, x, y + k, z) - ldz(p, g, x, y - k, z));
        gp[2] += c * (ldz(p, g, x, y, z + k) - ldz(p, g, x, y, z - k));
        gr[0] += c * (ldz(r, g, x + k, y, z) - ldz(r, g, x - k, y, z));
        gr[1] += c * (ldz(r, g, x, y + k, z) - ldz(r, g, x, y - k, z));
        gr[2] += c * (ldz(r, g, x, y, z + k) - ldz(r, g, x, y, z - k));
    }
    float st, ct, sp, cp;
    sincosf(__ldg(th + q), &st, &ct);
    sincosf(__ldg(ph + q), &sp, &cp);
    const float n0 = st * cp, n1 = st * sp, n2 = ct;
#pragma unroll
    for (int i = 0; i < 3; i++) { gp[i] *= g.ih; gr[i] *= g.ih; }
    const float wp = n0 * gp[0] + n1 * gp[1] + n2 * gp[2];
    const float wr = n0 * gr[0] + n1 * gr[1] + n2 * gr[2];
    ex[q] = gp[0] - n0 * wp;
    ey[q] = gp[1] - n1 * wp;
    ez[q] = gp[2] - n2 * wp;
    fx[q] = n0 * wr;
    fy[q] = n1 * wr;
    fz[q] = n2 * wr;
}

// pass 2; adjoint != 0 drops the coupling (already applied to zeta) and,
// if grad != NULL, adds the imaging term grad -= sum_f u_f^k dt^2 (H zeta)_f / m.
template <int M>
__global__ void __launch_bounds__(TZ *TY)
tti_update_kernel(GridDev g, FDW w, const float *__restrict__ ex, const float *__restrict__ ey,
                  const float *__restrict__ ez, const float *__restrict__ fx,
                  const float *__restrict__ fy, const float *__restrict__ fz,
                  const float *__restrict__ m, const float *__restrict__ eps,
                  const float *__restrict__ del, const float *__restrict__ pc,
                  const float *__restrict__ rc, float *__restrict__ pp, float *__restrict__ rp,
                  int adjoint, const float *__restrict__ up, const float *__restrict__ ur,
                  float *__restrict__ grad, int *flag, int check)
{
    const int z = blockIdx.x * TZ + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int x = blockIdx.z;
    if (z >= g.NZ || y >= g.NY) return;
    const long long q = gidx(g, x, y, z);
    float h0 = 0.f, hz = 0.f;
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const float c = w.c[k - 1];
        h0 += c * ((ldz(ex, g, x + k, y, z) - ldz(ex, g, x - k, y, z)) +
                   (ldz(ey, g, x, y + k, z) - ldz(ey, g, x, y - k, z)) +
                   (ldz(ez, g, x, y, z + k) - ldz(ez, g, x, y, z - k)));
        hz += c * ((ldz(fx, g, x + k, y, z) - ldz(fx, g, x - k, y, z)) +
                   (ldz(fy, g, x, y + k, z) - ldz(fy, g, x, y - k, z)) +
                   (ldz(fz, g, x, y, z + k) - ldz(fz, g, x, y, z - k)));
    }
    h0 *= g.ih;
    hz *= g.ih;
    float Lp, Lr;
    if (!adjoint) {
        const float a = 1.f + 2.f * __ldg(eps + q);
        const float s = sqrtf(1.f + 2.f * __ldg(del + q));
        Lp = a * h0 + s * hz;
        Lr = s * h0 + hz;
    } else {
        Lp = h0;
        Lr = hz;
    }
    const float mm = __ldg(m + q);
    const float sd = 0.5f * tti_sigma(g, x, y, z) * g.dt;
    const float A = mm * (1.f + sd), B = mm * (1.f - sd);
    const float dt2 = g.dt * g.dt;
    const float pn = (dt2 * Lp + 2.f * mm * __ldg(pc + q) - B * pp[q]) / A;
    const float rn = (dt2 * Lr + 2.f * mm * __ldg(rc + q) - B * rp[q]) / A;
    pp[q] = pn;
    rp[q] = rn;
    if (grad) grad[q] -= dt2 * (__ldg(up + q) * Lp + __ldg(ur + q) * Lr) / mm;
    if (check && !(isfinite(pn) && isfinite(rn))) atomicOr(flag, 1);
}

template <int M>
int launch(prop_s *P, float *const *S, bool adjoint, const float *up, const float *ur, float *grad)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, g.NX);
    const float *p = S[0], *r = S[1];
    if (adjoint) {
        k_tti_zeta(P, S[0], S[1], P->tmp[6], P->tmp[7]);
        p = P->tmp[6];
        r = P->tmp[7];
    }
    prof_begin(P, adjoint ? 1 : 0);
    tti_rot_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, p, r, P->th, P->ph, P->tmp[0], P->tmp[1],
                                                   P->tmp[2], P->tmp[3], P->tmp[4], P->tmp[5]);
    tti_update_kernel<M><<<grd, blk, 0, P->stream>>>(
        g, P->w, P->tmp[0], P->tmp[1], P->tmp[2], P->tmp[3], P->tmp[4], P->tmp[5], P->m, P->eps,
        P->del, S[0], S[1], S[2], S[3], adjoint ? 1 : 0, up, ur, grad, P->flag,
        P->d.check_nan);
    prof_end(P, adjoint ? 1 : 0);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

int tti_launch_step(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                    float *grad)
{
    switch (P->M) {
    case 2: return launch<2>(P, S, adjoint, img_p, img_r, grad);
    case 4: return launch<4>(P, S, adjoint, img_p, img_r, grad);
    case 6: return launch<6>(P, S, adjoint, img_p, img_r, grad);
    case 8: return launch<8>(P, S, adjoint, img_p, img_r, grad);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
