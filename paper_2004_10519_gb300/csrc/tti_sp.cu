// Staggered-pair variant of the TTI passes.  With P0 = I - n n^T and
// Pz = n n^T (pointwise), the composed centred operators of Sec. III-A are
//   H0 u = sum_{i,j} D_i (P0_ij D_j u),  Hz u = sum_{i,j} D_i (Pz_ij D_j u);
// here each diagonal term uses the staggered pair, D-_i (P_ii~ D+_i u), with
// P_ii~ the average of P_ii over the two nodes of the half point (the
// neighbour clamped at the last node), which leaves no checkerboard null
// vector; the cross terms i != j keep the centred D.  Both operators stay
// symmetric ((D+)^T = -D- and D^T = -D with zero extension), so the
// transposed step has the structure of the centred one: C applied before the
// stencil (zeta = C lam, kept by the update pass and the residual
// injection), imaging fused in the update pass.
//   pass 1: from (p, r) or zeta: the cross fluxes c0_i = sum_{j!=i} P0_ij D_j p,
//           cz_i = sum_{j!=i} Pz_ij D_j r and the diagonal fluxes at the half
//           points s0_i = P0_ii~ D+_i p, sz_i = Pz_ii~ D+_i r (12 fields);
//   pass 2: H0 p = sum_i (D_i c0_i + D-_i s0_i), Hz r likewise, coupling,
//           damped leapfrog (and zeta, imaging in the transposed step).
// One point per thread with read-only-cache loads (any NZ).
#include "common.cuh"

namespace {

constexpr int BZ = 32, BY = 8;

struct F12 {
    float *f[12];
};

WP_DEV float lz(const float *__restrict__ f, const GridDev &g, int x, int y, int z) { return ldz(f, g, x, y, z); }

template <int M>
__global__ void __launch_bounds__(BZ * BY)
tti_sp_rot(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
           const float *__restrict__ nxa, const float *__restrict__ nya, F12 o)
{
    const int z = blockIdx.x * BZ + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, x = blockIdx.z;
    if (z >= g.NZ || y >= g.NY) return;
    const long long q = gidx(g, x, y, z);
    float cp[3] = {0.f, 0.f, 0.f}, sp[3] = {0.f, 0.f, 0.f}, cr[3] = {0.f, 0.f, 0.f}, sr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int ex = a == 0, ey = a == 1, ez = a == 2;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const int xp = x + ex * k, yp = y + ey * k, zp = z + ez * k;
            const int xm = x - ex * k, ym = y - ey * k, zm = z - ez * k;
            const int xn = x - ex * (k - 1), yn = y - ey * (k - 1), zn = z - ez * (k - 1);
            const float pp = lz(p, g, xp, yp, zp), pm = lz(p, g, xm, ym, zm), pn = lz(p, g, xn, yn, zn);
            const float rp = lz(r, g, xp, yp, zp), rm = lz(r, g, xm, ym, zm), rn = lz(r, g, xn, yn, zn);
            cp[a] += w.c[k - 1] * (pp - pm);
            sp[a] += w.b[k - 1] * (pp - pn);
            cr[a] += w.c[k - 1] * (rp - rm);
            sr[a] += w.b[k - 1] * (rp - rn);
        }
        cp[a] *= g.ih;
        sp[a] *= g.ih;
        cr[a] *= g.ih;
        sr[a] *= g.ih;
    }
    const float n0 = __ldg(nxa + q), n1 = __ldg(nya + q);
    const float nv[3] = {n0, n1, sqrtf(fmaxf(0.f, 1.f - n0 * n0 - n1 * n1))};
    // n_i^2 at the node q + e_i (clamped): the other end of the half point
    const long long qx = gidx(g, min(x + 1, g.NX - 1), y, z), qy = gidx(g, x, min(y + 1, g.NY - 1), z),
                    qz = gidx(g, x, y, min(z + 1, g.NZ - 1));
    const float ax = __ldg(nxa + qx), by = __ldg(nya + qy);
    const float cx = __ldg(nxa + qz), cy = __ldg(nya + qz);
    const float n2n[3] = {ax * ax, by * by, fmaxf(0.f, 1.f - cx * cx - cy * cy)};
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float a0 = 0.f, az = 0.f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (j == i) continue;
            a0 += nv[j] * cp[j];
            az += nv[j] * cr[j];
        }
        const float ni2 = nv[i] * nv[i];
        o.f[i][q] = -nv[i] * a0;                                          // c0_i
        o.f[3 + i][q] = nv[i] * az;                                       // cz_i
        o.f[6 + i][q] = 0.5f * ((1.f - ni2) + (1.f - n2n[i])) * sp[i];   // s0_i
        o.f[9 + i][q] = 0.5f * (ni2 + n2n[i]) * sr[i];                    // sz_i
    }
}

template <int M, int ADJ, int GRAD>
__global__ void __launch_bounds__(BZ * BY)
tti_sp_upd(GridDev g, FDW w, F12 o, const float *__restrict__ m, const float *__restrict__ eps,
           const float *__restrict__ del, const float *__restrict__ p1, const float *__restrict__ r1,
           float *p0, float *r0, const float *__restrict__ up, const float *__restrict__ ur, float *grad,
           float *zp, float *zr, int *flag, int check)
{
    const int z = blockIdx.x * BZ + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, x = blockIdx.z;
    if (z >= g.NZ || y >= g.NY) return;
    const long long q = gidx(g, x, y, z);
    float h0 = 0.f, hz = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int ex = a == 0, ey = a == 1, ez = a == 2;
        const float *c0 = o.f[a], *cz = o.f[3 + a], *s0 = o.f[6 + a], *sz = o.f[9 + a];
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const int xp = x + ex * k, yp = y + ey * k, zp_ = z + ez * k;
            const int xm = x - ex * k, ym = y - ey * k, zm = z - ez * k;
            const int xh = x + ex * (k - 1), yh = y + ey * (k - 1), zh = z + ez * (k - 1);
            // D_i c (centred) + D-_i s (half -> node: s_{i+k-1} - s_{i-k})
            h0 += w.c[k - 1] * (lz(c0, g, xp, yp, zp_) - lz(c0, g, xm, ym, zm)) +
                  w.b[k - 1] * (lz(s0, g, xh, yh, zh) - lz(s0, g, xm, ym, zm));
            hz += w.c[k - 1] * (lz(cz, g, xp, yp, zp_) - lz(cz, g, xm, ym, zm)) +
                  w.b[k - 1] * (lz(sz, g, xh, yh, zh) - lz(sz, g, xm, ym, zm));
        }
    }
    h0 *= g.ih;
    hz *= g.ih;
    const float c1 = 1.f + 2.f * __ldg(eps + q), c2 = sqrtf(1.f + 2.f * __ldg(del + q));
    const float Lp = ADJ ? h0 : c1 * h0 + c2 * hz, Lr = ADJ ? hz : c2 * h0 + hz;
    const float dt2 = g.dt * g.dt, mm = __ldg(m + q);
    const float sd = 0.5f * g.dt * tti_sigma(g, x, y, z);
    const float A = mm * (1.f + sd), Bc = mm * (1.f - sd);
    const float pn = (dt2 * Lp + 2.f * mm * __ldg(p1 + q) - Bc * p0[q]) / A;
    const float rn = (dt2 * Lr + 2.f * mm * __ldg(r1 + q) - Bc * r0[q]) / A;
    p0[q] = pn;
    r0[q] = rn;
    if (ADJ) {
        zp[q] = c1 * pn + c2 * rn;
        zr[q] = c2 * pn + rn;
    }
    if (GRAD) grad[q] -= dt2 * (__ldg(up + q) * Lp + __ldg(ur + q) * Lr) / mm;
    if (check && !(isfinite(pn) && isfinite(rn))) atomicOr(flag, 1);
}

template <int M>
int launch(prop_s *P, float *const *S, bool adjoint, const float *up, const float *ur, float *grad)
{
    const GridDev &g = P->g;
    float *const *t = P->tmp;
    F12 o;
    for (int i = 0; i < 6; i++) o.f[i] = t[i];
    for (int i = 0; i < 6; i++) o.f[6 + i] = t[8 + i];
    dim3 blk(BZ, BY), grd((g.NZ + BZ - 1) / BZ, (g.NY + BY - 1) / BY, g.NX);
    // the rotation pass differentiates (p, r), or zeta = C lam (tmp[6], tmp[7])
    const float *rp_ = adjoint ? t[6] : S[0], *rr_ = adjoint ? t[7] : S[1];
    tti_sp_rot<M><<<grd, blk, 0, P->stream>>>(g, P->w, rp_, rr_, P->nrm[0], P->nrm[1], o);
    const int chk = P->d.check_nan;
    if (!adjoint)
        tti_sp_upd<M, 0, 0><<<grd, blk, 0, P->stream>>>(g, P->w, o, P->m, P->eps, P->del, S[0], S[1], S[2], S[3],
                                                        nullptr, nullptr, nullptr, nullptr, nullptr, P->flag, chk);
    else if (!grad)
        tti_sp_upd<M, 1, 0><<<grd, blk, 0, P->stream>>>(g, P->w, o, P->m, P->eps, P->del, S[0], S[1], S[2], S[3],
                                                        nullptr, nullptr, nullptr, t[6], t[7], P->flag, chk);
    else
        tti_sp_upd<M, 1, 1><<<grd, blk, 0, P->stream>>>(g, P->w, o, P->m, P->eps, P->del, S[0], S[1], S[2], S[3],
                                                        up, ur, grad, t[6], t[7], P->flag, chk);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// one TTI step with the staggered-pair operators (same contract as
// tti_launch_step; uses tmp[0..5], tmp[8..13] and zeta in tmp[6], tmp[7])
int tti_sp_launch(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r, float *grad)
{
    prof_begin(P, adjoint ? 1 : 0);
    int rc;
    switch (P->M) {
    case 2: rc = launch<2>(P, S, adjoint, img_p, img_r, grad); break;
    case 4: rc = launch<4>(P, S, adjoint, img_p, img_r, grad); break;
    case 6: rc = launch<6>(P, S, adjoint, img_p, img_r, grad); break;
    case 8: rc = launch<8>(P, S, adjoint, img_p, img_r, grad); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, adjoint ? 1 : 0);
    return rc;
}
