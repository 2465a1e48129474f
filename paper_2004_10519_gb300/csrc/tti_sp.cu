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
// Both passes stream along x over a 32(z) x 16(y) tile (any NZ): x
// derivatives from per-thread register queues, y and z derivatives from
// double-buffered shared planes whose halo loads are spread over the
// threads and issued one plane ahead.
#include "tile.cuh"

namespace {

using namespace tile;

struct F12 {
    float *f[12];
};

// pass 1 on (p, r) (forward) or (zeta_p, zeta_r) (transposed step)
template <int M>
__global__ void __launch_bounds__(NT, 1)
tti_sp_rot(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
           const float *__restrict__ nxa, const float *__restrict__ nya, F12 o, int xc)
{
    constexpr int Q = 2 * M + 1, SZ = PG<M>::size(2), C2 = PG<M>::cols(2);
    constexpr int S = (2 * PG<M>::nhalo(2) + NT - 1) / NT;
    extern __shared__ float sm[];               // [2 buffers][p, r][SZ]
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    HaloShare<M, 2, S> hs;
    hs.init([](int) { return 2; }, [](int k) { return k * SZ; }, tid);
    float qp[Q], qr[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qp[j] = lz(p, g, xa - M + j, y, z);
        qr[j] = lz(r, g, xa - M + j, y, z);
    }
    float np_, nr_, hv[S];
    auto fetch = [&](int x) {
        np_ = lz(p, g, x + M, y, z);
        nr_ = lz(r, g, x + M, y, z);
#pragma unroll
        for (int k = 0; k < S; k++) {
            const int f = hs.fld(k);
            hv[k] = f >= 0 ? lz(f ? r : p, g, x, y0 + hs.dy(k), z0 + hs.dz(k)) : 0.f;
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
            if (hs.fld(k) >= 0) sm[((x - xa) & 1) * 2 * SZ + hs.off[k]] = hv[k];
        __syncthreads();
        const long long q = act ? gidx(g, x, y, z) : 0;
        float n0 = 0.f, n1 = 0.f, ax = 0.f, by = 0.f, cx = 0.f, cy = 0.f;
        if (act) {
            n0 = __ldg(nxa + q);
            n1 = __ldg(nya + q);
            // the other node of each half point (clamped)
            ax = __ldg(nxa + gidx(g, min(x + 1, g.NX - 1), y, z));
            by = __ldg(nya + gidx(g, x, min(y + 1, g.NY - 1), z));
            const long long qz = gidx(g, x, y, min(z + 1, g.NZ - 1));
            cx = __ldg(nxa + qz);
            cy = __ldg(nya + qz);
        }
        if (x + 1 < xb) fetch(x + 1);
        if (act) {
            float cp[3] = {0.f, 0.f, 0.f}, cr[3] = {0.f, 0.f, 0.f}, tp[3] = {0.f, 0.f, 0.f}, tr[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1], b = w.b[k - 1];
                cp[0] += c * (qp[M + k] - qp[M - k]);
                cr[0] += c * (qr[M + k] - qr[M - k]);
                tp[0] += b * (qp[M + k] - qp[M - k + 1]);
                tr[0] += b * (qr[M + k] - qr[M - k + 1]);
                const float pyp = sp[ci + k * C2], pym = sp[ci - k * C2], pyn = sp[ci - (k - 1) * C2];
                const float ryp = sr[ci + k * C2], rym = sr[ci - k * C2], ryn = sr[ci - (k - 1) * C2];
                cp[1] += c * (pyp - pym);
                cr[1] += c * (ryp - rym);
                tp[1] += b * (pyp - pyn);
                tr[1] += b * (ryp - ryn);
                const float pzp = sp[ci + k], pzm = sp[ci - k], pzn = sp[ci - k + 1];
                const float rzp = sr[ci + k], rzm = sr[ci - k], rzn = sr[ci - k + 1];
                cp[2] += c * (pzp - pzm);
                cr[2] += c * (rzp - rzm);
                tp[2] += b * (pzp - pzn);
                tr[2] += b * (rzp - rzn);
            }
#pragma unroll
            for (int i = 0; i < 3; i++) {
                cp[i] *= g.ih;
                cr[i] *= g.ih;
                tp[i] *= g.ih;
                tr[i] *= g.ih;
            }
            const float nv[3] = {n0, n1, sqrtf(fmaxf(0.f, 1.f - n0 * n0 - n1 * n1))};
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
                o.f[6 + i][q] = 0.5f * ((1.f - ni2) + (1.f - n2n[i])) * tp[i];   // s0_i
                o.f[9 + i][q] = 0.5f * (ni2 + n2n[i]) * tr[i];                    // sz_i
            }
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qp[j] = qp[j + 1];
            qr[j] = qr[j + 1];
        }
    }
}

// pass 2.  planes: 0..3 = c0_y, cz_y, s0_y, sz_y (y halo); 4..7 = c0_z,
// cz_z, s0_z, sz_z (z halo); queues: c0_x, cz_x, s0_x, sz_x
template <int M, int ADJ, int GRAD>
__global__ void __launch_bounds__(NT, 1)
tti_sp_upd(GridDev g, FDW w, F12 o, const float *__restrict__ m, const float *__restrict__ eps,
           const float *__restrict__ del, const float *__restrict__ p1, const float *__restrict__ r1,
           float *p0, float *r0, const float *__restrict__ up, const float *__restrict__ ur, float *grad,
           float *zp, float *zr, int *flag, int check, int xc)
{
    constexpr int Q = 2 * M + 1, SY = PG<M>::size(0), SZZ = PG<M>::size(1);
    constexpr int C0 = PG<M>::cols(0);
    constexpr int BUF = 4 * SY + 4 * SZZ;
    constexpr int S = (4 * PG<M>::nhalo(0) + 4 * PG<M>::nhalo(1) + NT - 1) / NT;
    extern __shared__ float sm[];
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    // field k of the planes: o.f[pf(k)]; plane base k < 4: k SY, else 4 SY + (k - 4) SZZ
    auto pf = [](int k) { return k < 4 ? (k == 0 ? 1 : k == 1 ? 4 : k == 2 ? 7 : 10)
                                       : (k == 4 ? 2 : k == 5 ? 5 : k == 6 ? 8 : 11); };
    HaloShare<M, 8, S> hs;
    hs.init([](int k) { return k < 4 ? 0 : 1; }, [](int k) { return k < 4 ? k * SY : 4 * SY + (k - 4) * SZZ; },
            tid);
    float qc0[Q], qcz[Q], qs0[Q], qsz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qc0[j] = lz(o.f[0], g, xa - M + j, y, z);
        qcz[j] = lz(o.f[3], g, xa - M + j, y, z);
        qs0[j] = lz(o.f[6], g, xa - M + j, y, z);
        qsz[j] = lz(o.f[9], g, xa - M + j, y, z);
    }
    float nh[4], nown[8], hv[S];
    auto fetch = [&](int x) {
        nh[0] = lz(o.f[0], g, x + M, y, z);
        nh[1] = lz(o.f[3], g, x + M, y, z);
        nh[2] = lz(o.f[6], g, x + M, y, z);
        nh[3] = lz(o.f[9], g, x + M, y, z);
#pragma unroll
        for (int k = 0; k < 8; k++) nown[k] = lz(o.f[pf(k)], g, x, y, z);
#pragma unroll
        for (int k = 0; k < S; k++) {
            const int f = hs.fld(k);
            hv[k] = f >= 0 ? lz(o.f[pf(f)], g, x, y0 + hs.dy(k), z0 + hs.dz(k)) : 0.f;
        }
    };
    fetch(xa);
    const bool act = y < g.NY && z < g.NZ;
    const float dt2 = g.dt * g.dt, hdt = 0.5f * g.dt;
    const float syz = act ? __ldg(g.tab + g.NX + y) + __ldg(g.tab + g.NX + g.NY + z) : 0.f;
    const int i0 = PG<M>::inner(0, ty, tz), i1 = PG<M>::inner(1, ty, tz);
    for (int x = xa; x < xb; x++) {
        float *B = sm + ((x - xa) & 1) * BUF;
        qc0[Q - 1] = nh[0];
        qcz[Q - 1] = nh[1];
        qs0[Q - 1] = nh[2];
        qsz[Q - 1] = nh[3];
#pragma unroll
        for (int k = 0; k < 4; k++) B[k * SY + i0] = nown[k];
#pragma unroll
        for (int k = 0; k < 4; k++) B[4 * SY + k * SZZ + i1] = nown[4 + k];
#pragma unroll
        for (int k = 0; k < S; k++)
            if (hs.fld(k) >= 0) B[hs.off[k]] = hv[k];
        __syncthreads();
        const long long q = act ? gidx(g, x, y, z) : 0;
        float mm = 1.f, e_ = 0.f, d_ = 0.f, pc = 0.f, rc = 0.f, pq = 0.f, rq = 0.f;
        if (act) {
            mm = __ldg(m + q);
            e_ = __ldg(eps + q);
            d_ = __ldg(del + q);
            pc = __ldg(p1 + q);
            rc = __ldg(r1 + q);
            pq = p0[q];
            rq = r0[q];
        }
        if (x + 1 < xb) fetch(x + 1);
        if (act) {
            const float *yc0 = B, *ycz = B + SY, *ys0 = B + 2 * SY, *ysz = B + 3 * SY;
            const float *zc0 = B + 4 * SY, *zcz = zc0 + SZZ, *zs0 = zc0 + 2 * SZZ, *zsz = zc0 + 3 * SZZ;
            float h0 = 0.f, hz = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1], b = w.b[k - 1];
                // D_i c (centred) + D-_i s (half -> node: s_{i+k-1} - s_{i-k})
                h0 += c * ((qc0[M + k] - qc0[M - k]) + (yc0[i0 + k * C0] - yc0[i0 - k * C0]) +
                           (zc0[i1 + k] - zc0[i1 - k])) +
                      b * ((qs0[M + k - 1] - qs0[M - k]) + (ys0[i0 + (k - 1) * C0] - ys0[i0 - k * C0]) +
                           (zs0[i1 + k - 1] - zs0[i1 - k]));
                hz += c * ((qcz[M + k] - qcz[M - k]) + (ycz[i0 + k * C0] - ycz[i0 - k * C0]) +
                           (zcz[i1 + k] - zcz[i1 - k])) +
                      b * ((qsz[M + k - 1] - qsz[M - k]) + (ysz[i0 + (k - 1) * C0] - ysz[i0 - k * C0]) +
                           (zsz[i1 + k - 1] - zsz[i1 - k]));
            }
            h0 *= g.ih;
            hz *= g.ih;
            const float c1 = 1.f + 2.f * e_, c2 = sqrtf(1.f + 2.f * d_);
            const float Lp = ADJ ? h0 : c1 * h0 + c2 * hz, Lr = ADJ ? hz : c2 * h0 + hz;
            const float sd = hdt * (__ldg(g.tab + x) + syz);
            const float A = mm * (1.f + sd), Bc = mm * (1.f - sd);
            const float pn = (dt2 * Lp + 2.f * mm * pc - Bc * pq) / A;
            const float rn = (dt2 * Lr + 2.f * mm * rc - Bc * rq) / A;
            p0[q] = pn;
            r0[q] = rn;
            if (ADJ) {
                zp[q] = c1 * pn + c2 * rn;
                zr[q] = c2 * pn + rn;
            }
            if (GRAD) grad[q] -= dt2 * (__ldg(up + q) * Lp + __ldg(ur + q) * Lr) / mm;
            if (check && !(isfinite(pn) && isfinite(rn))) atomicOr(flag, 1);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qc0[j] = qc0[j + 1];
            qcz[j] = qcz[j + 1];
            qs0[j] = qs0[j + 1];
            qsz[j] = qsz[j + 1];
        }
    }
}

template <int M>
int launch(prop_s *P, float *const *S, bool adjoint, const float *up, const float *ur, float *grad)
{
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    float *const *t = P->tmp;
    F12 o;
    for (int i = 0; i < 6; i++) o.f[i] = t[i];
    for (int i = 0; i < 6; i++) o.f[6 + i] = t[8 + i];
    dim3 blk(FZ, FY, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    const size_t s1 = 2 * 2 * PG<M>::size(2) * sizeof(float);
    const size_t s2 = 2 * (4 * PG<M>::size(0) + 4 * PG<M>::size(1)) * sizeof(float);
    static const bool attr =
        (cudaFuncSetAttribute(tti_sp_rot<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1),
         cudaFuncSetAttribute(tti_sp_upd<M, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2),
         cudaFuncSetAttribute(tti_sp_upd<M, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2),
         cudaFuncSetAttribute(tti_sp_upd<M, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2), true);
    (void)attr;
    // the rotation pass differentiates (p, r), or zeta = C lam (tmp[6], tmp[7])
    const float *rp_ = adjoint ? t[6] : S[0], *rr_ = adjoint ? t[7] : S[1];
    tti_sp_rot<M><<<grd, blk, s1, P->stream>>>(g, P->w, rp_, rr_, P->nrm[0], P->nrm[1], o, xc);
    const int chk = P->d.check_nan;
    if (!adjoint)
        tti_sp_upd<M, 0, 0><<<grd, blk, s2, P->stream>>>(g, P->w, o, P->m, P->eps, P->del, S[0], S[1], S[2],
                                                         S[3], nullptr, nullptr, nullptr, nullptr, nullptr,
                                                         P->flag, chk, xc);
    else if (!grad)
        tti_sp_upd<M, 1, 0><<<grd, blk, s2, P->stream>>>(g, P->w, o, P->m, P->eps, P->del, S[0], S[1], S[2],
                                                         S[3], nullptr, nullptr, nullptr, t[6], t[7], P->flag,
                                                         chk, xc);
    else
        tti_sp_upd<M, 1, 1><<<grd, blk, s2, P->stream>>>(g, P->w, o, P->m, P->eps, P->del, S[0], S[1], S[2],
                                                         S[3], up, ur, grad, t[6], t[7], P->flag, chk, xc);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// one TTI step with the staggered-pair operators (same contract as
// tti_launch_step; uses tmp[0..5], tmp[8..13] and zeta in tmp[6], tmp[7]):
// the TMA-fed passes of tti_sp_tma.cu where NZ allows, else these
int tti_sp_launch(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r, float *grad)
{
    prof_begin(P, adjoint ? 1 : 0);
    int rc;
    if (tma_usable(P)) {
        rc = tti_sp_launch_tma(P, S, adjoint, img_p, img_r, grad);
        prof_end(P, adjoint ? 1 : 0);
        return rc;
    }
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
