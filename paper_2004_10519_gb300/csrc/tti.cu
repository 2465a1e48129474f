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
// Tiling: a CTA owns a TZ x TY tile of (y, z) columns and streams along x
// over a chunk of planes.  x-derivatives come from per-thread register
// queues, y- and z-derivatives from shared-memory planes with an M-point
// halo (loaded once per plane; zero outside the grid = zero extension).
#include "common.cuh"

namespace {

constexpr int TZ = 32, TY = 16, NT = TZ * TY;

WP_DEV float ldz2(const float *__restrict__ f, const GridDev &g, int x, int y, int z)
{
    return (x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ)
               ? __ldg(f + gidx(g, x, y, z)) : 0.f;
}

// value of the field(s) differentiated by pass 1 at (x,y,z): (p, r) or, in
// the adjoint, zeta = C (lam_p, lam_r)
template <bool ADJ>
WP_DEV void src_val(const GridDev &g, const float *__restrict__ p, const float *__restrict__ r,
                    const float *__restrict__ eps, const float *__restrict__ del, int x, int y, int z,
                    float &vp, float &vr)
{
    if (!(x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ)) {
        vp = vr = 0.f;
        return;
    }
    const long long q = gidx(g, x, y, z);
    const float a = __ldg(p + q), b = __ldg(r + q);
    if (!ADJ) {
        vp = a;
        vr = b;
    } else {
        const float c1 = 1.f + 2.f * __ldg(eps + q), c2 = sqrtf(1.f + 2.f * __ldg(del + q));
        vp = c1 * a + c2 * b;
        vr = c2 * a + b;
    }
}

template <int M, bool ADJ>
__global__ void __launch_bounds__(NT, 2)
tti_rot_kernel(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
               const float *__restrict__ eps, const float *__restrict__ del,
               const float *__restrict__ th, const float *__restrict__ ph,
               float *__restrict__ ex, float *__restrict__ ey, float *__restrict__ ez,
               float *__restrict__ fx, float *__restrict__ fy, float *__restrict__ fz, int xc)
{
    constexpr int HY = TY + 2 * M, HZ = TZ + 2 * M, Q = 2 * M + 1;
    __shared__ float sp[HY][HZ], sr[HY][HZ];
    const int tz = threadIdx.x, ty = threadIdx.y;
    const int z0 = blockIdx.x * TZ, y0 = blockIdx.y * TY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    float qp[Q], qr[Q];   // x - M .. x + M
#pragma unroll
    for (int j = 0; j < Q - 1; j++) src_val<ADJ>(g, p, r, eps, del, xa - M + j, y, z, qp[j], qr[j]);
    const bool act = y < g.NY && z < g.NZ;
    for (int x = xa; x < xb; x++) {
        src_val<ADJ>(g, p, r, eps, del, x + M, y, z, qp[Q - 1], qr[Q - 1]);
        __syncthreads();
        sp[ty + M][tz + M] = qp[M];
        sr[ty + M][tz + M] = qr[M];
        if (ty < M) {
            src_val<ADJ>(g, p, r, eps, del, x, y0 - M + ty, z, sp[ty][tz + M], sr[ty][tz + M]);
            src_val<ADJ>(g, p, r, eps, del, x, y0 + TY + ty, z, sp[ty + TY + M][tz + M], sr[ty + TY + M][tz + M]);
        }
        if (tz < M) {
            src_val<ADJ>(g, p, r, eps, del, x, y, z0 - M + tz, sp[ty + M][tz], sr[ty + M][tz]);
            src_val<ADJ>(g, p, r, eps, del, x, y, z0 + TZ + tz, sp[ty + M][tz + TZ + M], sr[ty + M][tz + TZ + M]);
        }
        __syncthreads();
        if (act) {
            float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f, gr0 = 0.f, gr1 = 0.f, gr2 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                gp0 += c * (qp[M + k] - qp[M - k]);
                gr0 += c * (qr[M + k] - qr[M - k]);
                gp1 += c * (sp[ty + M + k][tz + M] - sp[ty + M - k][tz + M]);
                gr1 += c * (sr[ty + M + k][tz + M] - sr[ty + M - k][tz + M]);
                gp2 += c * (sp[ty + M][tz + M + k] - sp[ty + M][tz + M - k]);
                gr2 += c * (sr[ty + M][tz + M + k] - sr[ty + M][tz + M - k]);
            }
            const long long q = gidx(g, x, y, z);
            float st, ct, sph, cph;
            sincosf(__ldg(th + q), &st, &ct);
            sincosf(__ldg(ph + q), &sph, &cph);
            const float n0 = st * cph, n1 = st * sph, n2 = ct;
            gp0 *= g.ih; gp1 *= g.ih; gp2 *= g.ih;
            gr0 *= g.ih; gr1 *= g.ih; gr2 *= g.ih;
            const float wp = n0 * gp0 + n1 * gp1 + n2 * gp2;
            const float wr = n0 * gr0 + n1 * gr1 + n2 * gr2;
            ex[q] = gp0 - n0 * wp;
            ey[q] = gp1 - n1 * wp;
            ez[q] = gp2 - n2 * wp;
            fx[q] = n0 * wr;
            fy[q] = n1 * wr;
            fz[q] = n2 * wr;
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qp[j] = qp[j + 1];
            qr[j] = qr[j + 1];
        }
    }
}

// pass 2; ADJ drops the coupling (already applied to zeta) and, if grad !=
// NULL, adds the imaging term grad -= sum_f u_f^k dt^2 (H zeta)_f / m.
template <int M, bool ADJ>
__global__ void __launch_bounds__(NT, 2)
tti_update_kernel(GridDev g, FDW w, const float *__restrict__ ex, const float *__restrict__ ey,
                  const float *__restrict__ ez, const float *__restrict__ fx,
                  const float *__restrict__ fy, const float *__restrict__ fz,
                  const float *__restrict__ m, const float *__restrict__ eps,
                  const float *__restrict__ del, const float *__restrict__ pc,
                  const float *__restrict__ rc, float *__restrict__ pp, float *__restrict__ rp,
                  const float *__restrict__ up, const float *__restrict__ ur,
                  float *__restrict__ grad, int *flag, int check, int xc)
{
    constexpr int HY = TY + 2 * M, HZ = TZ + 2 * M, Q = 2 * M + 1;
    __shared__ float sey[HY][TZ], sfy[HY][TZ], sez[TY][HZ], sfz[TY][HZ];
    const int tz = threadIdx.x, ty = threadIdx.y;
    const int z0 = blockIdx.x * TZ, y0 = blockIdx.y * TY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    const float *sx = g.tab, *sy = g.tab + g.NX, *sz = g.tab + g.NX + g.NY;   // damping per axis
    float qe[Q], qf[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qe[j] = ldz2(ex, g, xa - M + j, y, z);
        qf[j] = ldz2(fx, g, xa - M + j, y, z);
    }
    const bool act = y < g.NY && z < g.NZ;
    const float dt2 = g.dt * g.dt, hdt = 0.5f * g.dt;
    const float syz = act ? __ldg(sy + y) + __ldg(sz + z) : 0.f;
    for (int x = xa; x < xb; x++) {
        qe[Q - 1] = ldz2(ex, g, x + M, y, z);
        qf[Q - 1] = ldz2(fx, g, x + M, y, z);
        __syncthreads();
        sey[ty + M][tz] = ldz2(ey, g, x, y, z);
        sfy[ty + M][tz] = ldz2(fy, g, x, y, z);
        sez[ty][tz + M] = ldz2(ez, g, x, y, z);
        sfz[ty][tz + M] = ldz2(fz, g, x, y, z);
        if (ty < M) {
            sey[ty][tz] = ldz2(ey, g, x, y0 - M + ty, z);
            sfy[ty][tz] = ldz2(fy, g, x, y0 - M + ty, z);
            sey[ty + TY + M][tz] = ldz2(ey, g, x, y0 + TY + ty, z);
            sfy[ty + TY + M][tz] = ldz2(fy, g, x, y0 + TY + ty, z);
        }
        if (tz < M) {
            sez[ty][tz] = ldz2(ez, g, x, y, z0 - M + tz);
            sfz[ty][tz] = ldz2(fz, g, x, y, z0 - M + tz);
            sez[ty][tz + TZ + M] = ldz2(ez, g, x, y, z0 + TZ + tz);
            sfz[ty][tz + TZ + M] = ldz2(fz, g, x, y, z0 + TZ + tz);
        }
        __syncthreads();
        if (act) {
            float h0 = 0.f, hz = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                h0 += c * ((qe[M + k] - qe[M - k]) + (sey[ty + M + k][tz] - sey[ty + M - k][tz]) +
                           (sez[ty][tz + M + k] - sez[ty][tz + M - k]));
                hz += c * ((qf[M + k] - qf[M - k]) + (sfy[ty + M + k][tz] - sfy[ty + M - k][tz]) +
                           (sfz[ty][tz + M + k] - sfz[ty][tz + M - k]));
            }
            h0 *= g.ih;
            hz *= g.ih;
            const long long q = gidx(g, x, y, z);
            float Lp, Lr;
            if (!ADJ) {
                const float a = 1.f + 2.f * __ldg(eps + q);
                const float s = sqrtf(1.f + 2.f * __ldg(del + q));
                Lp = a * h0 + s * hz;
                Lr = s * h0 + hz;
            } else {
                Lp = h0;
                Lr = hz;
            }
            const float mm = __ldg(m + q);
            const float sd = hdt * (__ldg(sx + x) + syz);
            const float A = mm * (1.f + sd), B = mm * (1.f - sd);
            const float pn = (dt2 * Lp + 2.f * mm * __ldg(pc + q) - B * pp[q]) / A;
            const float rn = (dt2 * Lr + 2.f * mm * __ldg(rc + q) - B * rp[q]) / A;
            pp[q] = pn;
            rp[q] = rn;
            if (ADJ && grad) grad[q] -= dt2 * (__ldg(up + q) * Lp + __ldg(ur + q) * Lr) / mm;
            if (check && !(isfinite(pn) && isfinite(rn))) atomicOr(flag, 1);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qe[j] = qe[j + 1];
            qf[j] = qf[j + 1];
        }
    }
}

template <int M>
int launch(prop_s *P, float *const *S, bool adjoint, const float *up, const float *ur, float *grad)
{
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    prof_begin(P, adjoint ? 1 : 0);
    if (!adjoint) {
        tti_rot_kernel<M, false><<<grd, blk, 0, P->stream>>>(g, P->w, S[0], S[1], P->eps, P->del, P->th,
                                                             P->ph, t[0], t[1], t[2], t[3], t[4], t[5], xc);
        tti_update_kernel<M, false><<<grd, blk, 0, P->stream>>>(
            g, P->w, t[0], t[1], t[2], t[3], t[4], t[5], P->m, P->eps, P->del, S[0], S[1], S[2], S[3],
            nullptr, nullptr, nullptr, P->flag, P->d.check_nan, xc);
    } else {
        tti_rot_kernel<M, true><<<grd, blk, 0, P->stream>>>(g, P->w, S[0], S[1], P->eps, P->del, P->th,
                                                            P->ph, t[0], t[1], t[2], t[3], t[4], t[5], xc);
        tti_update_kernel<M, true><<<grd, blk, 0, P->stream>>>(
            g, P->w, t[0], t[1], t[2], t[3], t[4], t[5], P->m, P->eps, P->del, S[0], S[1], S[2], S[3],
            up, ur, grad, P->flag, P->d.check_nan, xc);
    }
    prof_end(P, adjoint ? 1 : 0);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

int tti_launch_step(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                    float *grad)
{
    return tma_usable(P) ? tti_launch_tma(P, S, adjoint, img_p, img_r, grad)
                         : tti_launch_fast(P, S, adjoint, img_p, img_r, grad);
}

// first tiled form (loads of plane x issued after the previous barrier);
// kept as the comparison point of the pipelined passes in tti_fast.cu
int tti_launch_tiled(prop_s *P, float *const *S, bool adjoint, const float *img_p,
                     const float *img_r, float *grad)
{
    switch (P->M) {
    case 2: return launch<2>(P, S, adjoint, img_p, img_r, grad);
    case 4: return launch<4>(P, S, adjoint, img_p, img_r, grad);
    case 6: return launch<6>(P, S, adjoint, img_p, img_r, grad);
    case 8: return launch<8>(P, S, adjoint, img_p, img_r, grad);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

// x-chunk length: enough CTAs for several waves of 2 CTAs per SM
int stencil_xchunk(const GridDev &g, int sms)
{
    const long long tiles = (long long)((g.NZ + TZ - 1) / TZ) * ((g.NY + TY - 1) / TY);
    const long long slots = 2LL * sms;
    long long chunks = std::max(1LL, (5 * slots + tiles - 1) / tiles);
    // round so that the CTA count is close to a whole number of waves
    long long best = chunks, bestw = 1 << 30;
    for (long long c = std::max(1LL, chunks - 3); c <= chunks + 3; c++) {
        long long ctas = tiles * c, rem = ctas % slots;
        long long waste = rem ? slots - rem : 0;
        if (waste < bestw) { bestw = waste; best = c; }
    }
    int xc = (int)((g.NX + best - 1) / best);
    return std::max(xc, std::min(g.NX, 8));
}
