// Pipelined TTI step passes (Sec. III-A; operator definitions in tti.cu).
//
//   pass 1: e_i = D_i p - n_i (n . D p),  f_i = n_i (n . D r)
//           (adjoint: D applied to zeta = C lam, formed while loading)
//   pass 2: H0 p = sum_i D_i e_i, Hz r = sum_i D_i f_i, coupling C (forward
//           only), damped leapfrog; adjoint: fused imaging
//           grad -= sum_f u_f^k dt^2 (H zeta)_f / m.
// Imaging of eps, delta, theta, phi (prop_gradient_aniso) on these passes:
// pass 1 in its RAW mode writes D p, D r unprojected; pass 2 in mode
// ADJ = 2 takes no step and accumulates the coupling terms with lam^{n+1}
// (see tti_image_aniso_fast).
// Each pass streams along x over a 32(z) x 16(y) tile.  The loads of plane
// x+1 (queue heads, own interior values, an even share of the halo) are in
// flight while plane x is computed from double-buffered shared planes.
#include "tile.cuh"

namespace {

using namespace tile;

template <bool ADJ>
WP_DEV void src_pair(const GridDev &g, const float *__restrict__ p, const float *__restrict__ r,
                     const float *__restrict__ eps, const float *__restrict__ del, int x, int y,
                     int z, float &vp, float &vr)
{
    if (!inside(g, x, y, z)) {
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

template <int M, int ADJ, bool RAW = false>
__global__ void __launch_bounds__(NT, 2)
tti_rot_p(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
          const float *__restrict__ eps, const float *__restrict__ del, const float *__restrict__ nxa,
          const float *__restrict__ nya, float *__restrict__ ex, float *__restrict__ ey,
          float *__restrict__ ez, float *__restrict__ fx, float *__restrict__ fy,
          float *__restrict__ fz, int xc)
{
    constexpr int Q = 2 * M + 1, SZ = PG<M>::size(2), C2 = PG<M>::cols(2);
    constexpr int S = (PG<M>::nhalo(2) + NT - 1) / NT;
    extern __shared__ float sm[];               // [2 buffers][p, r][SZ]
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    HaloShare<M, 1, S> hs;
    hs.init([](int) { return 2; }, [](int) { return 0; }, tid);
    float qp[Q], qr[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) src_pair<ADJ>(g, p, r, eps, del, xa - M + j, y, z, qp[j], qr[j]);
    float np_, nr_, hp[S], hr[S];
    auto fetch = [&](int x) {
        src_pair<ADJ>(g, p, r, eps, del, x + M, y, z, np_, nr_);
#pragma unroll
        for (int k = 0; k < S; k++) {
            hp[k] = hr[k] = 0.f;
            if (hs.fld(k) >= 0)
                src_pair<ADJ>(g, p, r, eps, del, x, y0 + hs.dy(k), z0 + hs.dz(k), hp[k], hr[k]);
        }
    };
    fetch(xa);
    const bool act = y < g.NY && z < g.NZ;
    const int ci = PG<M>::inner(2, ty, tz);
    for (int x = xa; x < xb; x++) {
        float *sp = sm + ((x - xa) & 1) * 2 * SZ, *sr = sp + SZ;
        qp[Q - 1] = np_;
        qr[Q - 1] = nr_;
        sp[ci] = qp[M];
        sr[ci] = qr[M];
#pragma unroll
        for (int k = 0; k < S; k++)
            if (hs.fld(k) >= 0) {
                sp[hs.off[k]] = hp[k];
                sr[hs.off[k]] = hr[k];
            }
        __syncthreads();
        float n0 = 0.f, n1 = 0.f;
        const long long q = act ? gidx(g, x, y, z) : 0;
        if (act) {
            n0 = __ldg(nxa + q);
            n1 = __ldg(nya + q);
        }
        if (x + 1 < xb) fetch(x + 1);
        if (act) {
            float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f, gr0 = 0.f, gr1 = 0.f, gr2 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                gp0 += c * (qp[M + k] - qp[M - k]);
                gr0 += c * (qr[M + k] - qr[M - k]);
                gp1 += c * (sp[ci + k * C2] - sp[ci - k * C2]);
                gr1 += c * (sr[ci + k * C2] - sr[ci - k * C2]);
                gp2 += c * (sp[ci + k] - sp[ci - k]);
                gr2 += c * (sr[ci + k] - sr[ci - k]);
            }
            // symmetry axis from the precomputed (n_x, n_y), n_z >= 0
            const float n2 = sqrtf(fmaxf(0.f, 1.f - n0 * n0 - n1 * n1));
            gp0 *= g.ih; gp1 *= g.ih; gp2 *= g.ih;
            gr0 *= g.ih; gr1 *= g.ih; gr2 *= g.ih;
            if constexpr (RAW) {
                ex[q] = gp0;
                ey[q] = gp1;
                ez[q] = gp2;
                fx[q] = gr0;
                fy[q] = gr1;
                fz[q] = gr2;
            } else {
            const float wp = n0 * gp0 + n1 * gp1 + n2 * gp2;
            const float wr = n0 * gr0 + n1 * gr1 + n2 * gr2;
            ex[q] = gp0 - n0 * wp;
            ey[q] = gp1 - n1 * wp;
            ez[q] = gp2 - n2 * wp;
            fx[q] = n0 * wr;
            fy[q] = n1 * wr;
            fz[q] = n2 * wr;
            }
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qp[j] = qp[j + 1];
            qr[j] = qr[j + 1];
        }
    }
}

// fields: 0 e_y, 1 f_y (y halo); 2 e_z, 3 f_z (z halo)
template <int M, int ADJ>
__global__ void __launch_bounds__(NT, 2)
tti_upd_p(GridDev g, FDW w, const float *__restrict__ ex, const float *__restrict__ ey,
          const float *__restrict__ ez, const float *__restrict__ fx, const float *__restrict__ fy,
          const float *__restrict__ fz, const float *__restrict__ m, const float *__restrict__ eps,
          const float *__restrict__ del, const float *__restrict__ pc, const float *__restrict__ rc,
          float *__restrict__ pp, float *__restrict__ rp, const float *__restrict__ up,
          const float *__restrict__ ur, float *__restrict__ grad, int *flag, int check, int xc)
{
    constexpr int Q = 2 * M + 1, SY = PG<M>::size(0), SZZ = PG<M>::size(1);
    constexpr int C0 = PG<M>::cols(0), C1 = PG<M>::cols(1);
    constexpr int BUF = 2 * SY + 2 * SZZ;
    constexpr int S = (2 * PG<M>::nhalo(0) + 2 * PG<M>::nhalo(1) + NT - 1) / NT;
    extern __shared__ float sm[];
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    HaloShare<M, 4, S> hs;
    hs.init([](int k) { return k < 2 ? 0 : 1; },
            [](int k) { return k == 0 ? 0 : k == 1 ? SY : k == 2 ? 2 * SY : 2 * SY + SZZ; }, tid);
    auto pick = [&](int k) { return k == 0 ? ey : k == 1 ? fy : k == 2 ? ez : fz; };
    float qe[Q], qf[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qe[j] = lz(ex, g, xa - M + j, y, z);
        qf[j] = lz(fx, g, xa - M + j, y, z);
    }
    float ne, nf, ney, nfy, nez, nfz, hv[S];
    auto fetch = [&](int x) {
        ne = lz(ex, g, x + M, y, z);
        nf = lz(fx, g, x + M, y, z);
        ney = lz(ey, g, x, y, z);
        nfy = lz(fy, g, x, y, z);
        nez = lz(ez, g, x, y, z);
        nfz = lz(fz, g, x, y, z);
#pragma unroll
        for (int k = 0; k < S; k++) {
            const int f = hs.fld(k);
            hv[k] = f >= 0 ? lz(pick(f), g, x, y0 + hs.dy(k), z0 + hs.dz(k)) : 0.f;
        }
    };
    fetch(xa);
    const bool act = y < g.NY && z < g.NZ;
    const float *sx = g.tab, *sy = g.tab + g.NX, *sz = g.tab + g.NX + g.NY;
    const float dt2 = g.dt * g.dt, hdt = 0.5f * g.dt;
    const float syz = act ? __ldg(sy + y) + __ldg(sz + z) : 0.f;
    const int i0 = PG<M>::inner(0, ty, tz), i1 = PG<M>::inner(1, ty, tz);
    for (int x = xa; x < xb; x++) {
        float *B = sm + ((x - xa) & 1) * BUF;
        qe[Q - 1] = ne;
        qf[Q - 1] = nf;
        B[i0] = ney;
        B[SY + i0] = nfy;
        B[2 * SY + i1] = nez;
        B[2 * SY + SZZ + i1] = nfz;
#pragma unroll
        for (int k = 0; k < S; k++)
            if (hs.fld(k) >= 0) B[hs.off[k]] = hv[k];
        __syncthreads();
        const long long q = act ? gidx(g, x, y, z) : 0;
        float mm = 1.f, e_ = 0.f, d_ = 0.f, p1 = 0.f, r1 = 0.f, p0 = 0.f, r0 = 0.f;
        if (act) {
            if (ADJ != 2) mm = __ldg(m + q);
            if (ADJ != 1) d_ = __ldg(del + q);
            if (ADJ == 0) e_ = __ldg(eps + q);
            p1 = __ldg(pc + q);
            r1 = __ldg(rc + q);
            p0 = pp[q];
            r0 = rp[q];
        }
        if (x + 1 < xb) fetch(x + 1);
        if (act) {
            const float *sey = B, *sfy = B + SY, *sez = B + 2 * SY, *sfz = B + 2 * SY + SZZ;
            float h0 = 0.f, hz = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                h0 += c * ((qe[M + k] - qe[M - k]) + (sey[i0 + k * C0] - sey[i0 - k * C0]) +
                           (sez[i1 + k] - sez[i1 - k]));
                hz += c * ((qf[M + k] - qf[M - k]) + (sfy[i0 + k * C0] - sfy[i0 - k * C0]) +
                           (sfz[i1 + k] - sfz[i1 - k]));
            }
            h0 *= g.ih;
            hz *= g.ih;
            if (ADJ == 2) {
                // imaging of the coupling with lam^{n+1} = (p1, r1) and the
                // forward field's H0 p^n, Hz r^n: g_eps (pp) += 2 dt^2
                // lam_p H0 p^n, g_delta (rp) += dt^2 (lam_p Hz r^n + lam_r
                // H0 p^n) / sqrt(1 + 2 delta)
                pp[q] = p0 + 2.f * dt2 * p1 * h0;
                rp[q] = r0 + dt2 * (p1 * hz + r1 * h0) / sqrtf(1.f + 2.f * d_);
            } else {
            float Lp, Lr;
            if (!ADJ) {
                const float a = 1.f + 2.f * e_, s = sqrtf(1.f + 2.f * d_);
                Lp = a * h0 + s * hz;
                Lr = s * h0 + hz;
            } else {
                Lp = h0;
                Lr = hz;
            }
            const float sd = hdt * (__ldg(sx + x) + syz);
            const float A = mm * (1.f + sd), Bc = mm * (1.f - sd);
            const float pn = (dt2 * Lp + 2.f * mm * p1 - Bc * p0) / A;
            const float rn = (dt2 * Lr + 2.f * mm * r1 - Bc * r0) / A;
            pp[q] = pn;
            rp[q] = rn;
            if (ADJ && grad) grad[q] -= dt2 * (__ldg(up + q) * Lp + __ldg(ur + q) * Lr) / mm;
            if (check && !(isfinite(pn) && isfinite(rn))) atomicOr(flag, 1);
            }
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qe[j] = qe[j + 1];
            qf[j] = qf[j + 1];
        }
    }
}

template <int M, int ADJ>
int launch(prop_s *P, float *const *S, const float *up, const float *ur, float *grad)
{
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(FZ, FY, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    const size_t s1 = 2 * 2 * PG<M>::size(2) * sizeof(float);
    const size_t s2 = 2 * (2 * PG<M>::size(0) + 2 * PG<M>::size(1)) * sizeof(float);
    static const bool attr = (cudaFuncSetAttribute(tti_rot_p<M, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1),
                              cudaFuncSetAttribute(tti_upd_p<M, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2), true);
    (void)attr;
    prof_begin(P, ADJ ? 1 : 0);
    tti_rot_p<M, ADJ><<<grd, blk, s1, P->stream>>>(g, P->w, S[0], S[1], P->eps, P->del, P->nrm[0], P->nrm[1],
                                                   t[0], t[1], t[2], t[3], t[4], t[5], xc);
    tti_upd_p<M, ADJ><<<grd, blk, s2, P->stream>>>(g, P->w, t[0], t[1], t[2], t[3], t[4], t[5], P->m,
                                                   P->eps, P->del, S[0], S[1], S[2], S[3], up, ur,
                                                   grad, P->flag, P->d.check_nan, xc);
    prof_end(P, ADJ ? 1 : 0);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

// eps, delta (and theta, phi) imaging of one transposed step on the
// pipelined passes: the rotation pass on the forward field (up, ur), the
// update pass in its imaging mode with lam = (lp, lr); with gax, zeta = C lam
// into tmp[6], tmp[7], raw derivatives of zeta (tmp[0..5]) and of the
// forward field (tmp[8..13]) and the pointwise axis term
template <int M>
int image_aniso(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr, float *ge,
                float *gd, float *const *gax)
{
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(FZ, FY, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    const size_t s1 = 2 * 2 * PG<M>::size(2) * sizeof(float);
    const size_t s2 = 2 * (2 * PG<M>::size(0) + 2 * PG<M>::size(1)) * sizeof(float);
    static const bool attr =
        (cudaFuncSetAttribute(tti_rot_p<M, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1),
         cudaFuncSetAttribute(tti_rot_p<M, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1),
         cudaFuncSetAttribute(tti_upd_p<M, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2), true);
    (void)attr;
    tti_rot_p<M, 0><<<grd, blk, s1, P->stream>>>(g, P->w, up, ur, P->eps, P->del, P->nrm[0], P->nrm[1], t[0], t[1],
                                                 t[2], t[3], t[4], t[5], xc);
    tti_upd_p<M, 2><<<grd, blk, s2, P->stream>>>(g, P->w, t[0], t[1], t[2], t[3], t[4], t[5], P->m, P->eps, P->del,
                                                 lp, lr, ge, gd, nullptr, nullptr, nullptr, P->flag, 0, xc);
    P->kern_launches += 2;
    if (gax) {
        k_tti_zeta(P, lp, lr, t[6], t[7]);
        tti_rot_p<M, 0, true><<<grd, blk, s1, P->stream>>>(g, P->w, t[6], t[7], P->eps, P->del, P->nrm[0],
                                                           P->nrm[1], t[0], t[1], t[2], t[3], t[4], t[5], xc);
        tti_rot_p<M, 0, true><<<grd, blk, s1, P->stream>>>(g, P->w, up, ur, P->eps, P->del, P->nrm[0], P->nrm[1],
                                                           t[8], t[9], t[10], t[11], t[12], t[13], xc);
        P->kern_launches += 2;
        const float *dz[6] = {t[0], t[1], t[2], t[3], t[4], t[5]}, *du[6] = {t[8], t[9], t[10], t[11], t[12], t[13]};
        tti_axis_image_launch(P, dz, du, gax);
    }
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

int tti_image_aniso_fast(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr,
                         float *ge, float *gd, float *const *gax)
{
    switch (P->M) {
    case 2: return image_aniso<2>(P, up, ur, lp, lr, ge, gd, gax);
    case 4: return image_aniso<4>(P, up, ur, lp, lr, ge, gd, gax);
    case 6: return image_aniso<6>(P, up, ur, lp, lr, ge, gd, gax);
    case 8: return image_aniso<8>(P, up, ur, lp, lr, ge, gd, gax);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

int tti_launch_fast(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                    float *grad)
{
    switch (P->M) {
    case 2: return adjoint ? launch<2, 1>(P, S, img_p, img_r, grad) : launch<2, 0>(P, S, img_p, img_r, grad);
    case 4: return adjoint ? launch<4, 1>(P, S, img_p, img_r, grad) : launch<4, 0>(P, S, img_p, img_r, grad);
    case 6: return adjoint ? launch<6, 1>(P, S, img_p, img_r, grad) : launch<6, 0>(P, S, img_p, img_r, grad);
    case 8: return adjoint ? launch<8, 1>(P, S, img_p, img_r, grad) : launch<8, 0>(P, S, img_p, img_r, grad);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
