// Staggered-pair TTI passes fed by the Tensor Memory Accelerator (sm_103a).
//
// Same operators as the pipelined passes of tti_sp.cu (Sec. III-A with the
// diagonal terms D-_i (P_ii~ D+_i u), P_ii~ the two-node average of P_ii, the
// cross terms centred), on the plane ring of the other TMA-fed passes: a
// 32(z) x 16(y) tile streamed along x, two z points per consumer thread, a
// producer warp keeping three planes in flight, every wait bounded.
//   pass 1: (p, r) or zeta -> the twelve fluxes c0_i, cz_i (nodes) and
//           s0_i, sz_i (half points i+1/2, stored at index i);
//   pass 2: H0 p = sum_i (D_i c0_i + D-_i s0_i), Hz r likewise, coupling,
//           damped leapfrog (zeta and imaging in the transposed step).
// In pass 2 the x-derivatives of the four x fluxes are pushed into two
// queues of partial sums (H0 and Hz at planes x .. x+2M) as each plane's
// fluxes arrive, instead of holding four queues of inputs: half the queue
// registers for the same multiply-adds.
// Gradients w.r.t. eps and delta image the coupling with pass 2 in a mode
// without the step; the tilt/azimuth term adds, to the centred form's, the
// half-point products of the staggered diagonal terms (formed with the
// centred derivatives in the TMA rotation pass's mode 2, tti_raw_half_tma,
// then tti_axis_image_sp).
#include "tma.cuh"

namespace {

// ---------------------------------------------------------------------------
// pass 1.  stage: [p rect] [r rect] [queue heads p, r (x+M)] [n_x, n_y +1
// boxes (plane x)] [n_x (plane x+1, clamped)]
// ---------------------------------------------------------------------------
template <int M>
struct SRL {
    using B = BX<M>;
    static constexpr int OP = 0, OR = B::RS, OQ = 2 * B::RS, ONX = OQ + 2 * IS, ONY = ONX + B::PS,
                         OXN = ONY + B::PS, SZ = OXN + IS;
    static constexpr uint32_t BYTES = 4u * (2 * B::RR * B::RC + 2 * B::PR * B::PC + 3 * IS);
};

struct SRMaps {
    CUtensorMap p, r, qp, qr, nx1, ny1, nxi;
};

struct F12 {
    float *f[12];
};

template <int M>
__global__ void __launch_bounds__(NTP, M <= 6 ? 2 : 1)
tti_sp_rot_tma(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
               const __grid_constant__ SRMaps mp, F12 o, int xc, int *err)
{
    using L = SRL<M>;
    using B = BX<M>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, lane = (ty * TZ2 + tz) & 31;
    const bool lead = ty == 0 && tz == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + 2 * tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        uint64_t *bar = &bars[st];
        mbar_expect(bar, L::BYTES);
        tma3(S + L::OP, &mp.p, z0 - B::MZ, y0 - M, x, bar);
        tma3(S + L::OR, &mp.r, z0 - B::MZ, y0 - M, x, bar);
        tma3(S + L::OQ, &mp.qp, z0, y0, x + M, bar);                  // beyond NX: zeros
        tma3(S + L::OQ + IS, &mp.qr, z0, y0, x + M, bar);
        tma3(S + L::ONX, &mp.nx1, z0, y0, x, bar);
        tma3(S + L::ONY, &mp.ny1, z0, y0, x, bar);
        tma3(S + L::OXN, &mp.nxi, z0, y0, min(x + 1, g.NX - 1), bar);
    };
    Ring R(bars);
    if (lead) {
        R.init();
        ck_begin(g.N, err);
    }
    __syncthreads();
    if (ty >= FY) {                                       // producer warp
        if (lane == 0) R.produce(xa, nit, issue, err);
        return;
    }
    const bool act = y < g.NY && z < g.NZ;
    const unsigned pl = (unsigned)g.NY * (unsigned)g.NZ;
    const unsigned q0 = act ? (unsigned)y * g.NZ + z : 0u;
    const float2 Z2 = make_float2(0.f, 0.f);
    float2 qp[Q], qr[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        const int xq = xa - M + j;
        const bool in = act && xq >= 0 && xq < g.NX;
        qp[j] = in ? ldg2(p, xq * pl + q0) : Z2;
        qr[j] = in ? ldg2(r, xq * pl + q0) : Z2;
    }
    const int cy = ty + M, cz = B::MZ + 2 * tz, c2 = 2 * tz, ii = ty * FZ + c2;
    const int ci = cy * B::RC + cz;
    // the other node of each half point, clamped at the last node: row y+1,
    // and column z+2 for the second point (z+1 is the first point's)
    const int yb1 = y + 1 < g.NY ? ty + 1 : ty;
    const int zb2 = z + 2 < g.NZ ? c2 + 2 : c2 + 1;
    for (int x = xa; x < xb; x++) {
        if (!__all_sync(0xffffffffu, R.wait_full())) {
            if (lane == 0) atomicOr(err, 2);
            return;
        }
        const float *S = sm + R.st * L::SZ;
        qp[Q - 1] = lds2(S + L::OQ + ii);
        qr[Q - 1] = lds2(S + L::OQ + IS + ii);
        if (act) {
            const float *sp = S + L::OP, *sr = S + L::OR;
            // centred D_i (cp, cr) and staggered D+_i (tp, tr), both points
            float2 cp[3] = {Z2, Z2, Z2}, cr[3] = {Z2, Z2, Z2}, tp[3] = {Z2, Z2, Z2}, tr[3] = {Z2, Z2, Z2};
            {
                float2 prp = lds2(sp + ci), prr = lds2(sr + ci);   // row y: the y+1-k row of k = 1
#pragma unroll
                for (int k = 1; k <= M; k++) {
                    const float2 c = f2s(w.c[k - 1]), b = f2s(w.b[k - 1]);
                    cp[0] = f2fma(c, f2sub(qp[M + k], qp[M - k]), cp[0]);
                    cr[0] = f2fma(c, f2sub(qr[M + k], qr[M - k]), cr[0]);
                    tp[0] = f2fma(b, f2sub(qp[M + k], qp[M - k + 1]), tp[0]);
                    tr[0] = f2fma(b, f2sub(qr[M + k], qr[M - k + 1]), tr[0]);
                    const float2 pyp = lds2(sp + ci + k * B::RC), pym = lds2(sp + ci - k * B::RC);
                    const float2 ryp = lds2(sr + ci + k * B::RC), rym = lds2(sr + ci - k * B::RC);
                    cp[1] = f2fma(c, f2sub(pyp, pym), cp[1]);
                    cr[1] = f2fma(c, f2sub(ryp, rym), cr[1]);
                    tp[1] = f2fma(b, f2sub(pyp, prp), tp[1]);
                    tr[1] = f2fma(b, f2sub(ryp, prr), tr[1]);
                    prp = pym;
                    prr = rym;
                }
            }
            {
                float wv[2 * M + 2];
                zwin<M>(sp + cy * B::RC, cz, wv);
#pragma unroll
                for (int k = 1; k <= M; k++) {
                    const float2 c = f2s(w.c[k - 1]), b = f2s(w.b[k - 1]);
                    cp[2] = f2fma(c, make_float2(wv[M + k] - wv[M - k], wv[M + k + 1] - wv[M - k + 1]), cp[2]);
                    tp[2] = f2fma(b, make_float2(wv[M + k] - wv[M - k + 1], wv[M + k + 1] - wv[M - k + 2]), tp[2]);
                }
                zwin<M>(sr + cy * B::RC, cz, wv);
#pragma unroll
                for (int k = 1; k <= M; k++) {
                    const float2 c = f2s(w.c[k - 1]), b = f2s(w.b[k - 1]);
                    cr[2] = f2fma(c, make_float2(wv[M + k] - wv[M - k], wv[M + k + 1] - wv[M - k + 1]), cr[2]);
                    tr[2] = f2fma(b, make_float2(wv[M + k] - wv[M - k + 1], wv[M + k + 1] - wv[M - k + 2]), tr[2]);
                }
            }
            const float2 ih = f2s(g.ih);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                cp[i] = f2mul(cp[i], ih);
                cr[i] = f2mul(cr[i], ih);
                tp[i] = f2mul(tp[i], ih);
                tr[i] = f2mul(tr[i], ih);
            }
            const float *snx = S + L::ONX, *sny = S + L::ONY;
            const float2 nx0 = lds2(snx + ty * B::PC + c2), ny0 = lds2(sny + ty * B::PC + c2);
            const float2 axn = lds2(S + L::OXN + ii);                        // n_x at x+1
            const float2 byn = lds2(sny + yb1 * B::PC + c2);                 // n_y at y+1
            const float zx[2] = {nx0.y, snx[ty * B::PC + zb2]};             // n at z+1
            const float zy[2] = {ny0.y, sny[ty * B::PC + zb2]};
            const float NX0[2] = {nx0.x, nx0.y}, NY0[2] = {ny0.x, ny0.y};
            const float AX[2] = {axn.x, axn.y}, BY[2] = {byn.x, byn.y};
            float out[12][2];
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const float cpv[3] = {s ? cp[0].y : cp[0].x, s ? cp[1].y : cp[1].x, s ? cp[2].y : cp[2].x};
                const float crv[3] = {s ? cr[0].y : cr[0].x, s ? cr[1].y : cr[1].x, s ? cr[2].y : cr[2].x};
                const float tpv[3] = {s ? tp[0].y : tp[0].x, s ? tp[1].y : tp[1].x, s ? tp[2].y : tp[2].x};
                const float trv[3] = {s ? tr[0].y : tr[0].x, s ? tr[1].y : tr[1].x, s ? tr[2].y : tr[2].x};
                const float n0 = NX0[s], n1 = NY0[s];
                const float nv[3] = {n0, n1, sqrtf(fmaxf(0.f, 1.f - n0 * n0 - n1 * n1))};
                const float n2n[3] = {AX[s] * AX[s], BY[s] * BY[s], fmaxf(0.f, 1.f - zx[s] * zx[s] - zy[s] * zy[s])};
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    float a0 = 0.f, az = 0.f;
#pragma unroll
                    for (int j = 0; j < 3; j++) {
                        if (j == i) continue;
                        a0 += nv[j] * cpv[j];
                        az += nv[j] * crv[j];
                    }
                    const float ni2 = nv[i] * nv[i];
                    out[i][s] = -nv[i] * a0;                                           // c0_i
                    out[3 + i][s] = nv[i] * az;                                        // cz_i
                    out[6 + i][s] = 0.5f * ((1.f - ni2) + (1.f - n2n[i])) * tpv[i];   // s0_i
                    out[9 + i][s] = 0.5f * (ni2 + n2n[i]) * trv[i];                    // sz_i
                }
            }
            const unsigned q = x * pl + q0;
#pragma unroll
            for (int f = 0; f < 12; f++) st2(o.f[f], q, out[f][0], out[f][1]);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qp[j] = qp[j + 1];
            qr[j] = qr[j + 1];
        }
        R.release(lane);
    }
}

// ---------------------------------------------------------------------------
// pass 2.  stage: [c0_y, cz_y, s0_y, sz_y (y boxes)] [c0_z, cz_z, s0_z, sz_z
// (z boxes)] [heads c0_x, cz_x (x+M), s0_x, sz_x (x+M-1)] [m, p^n, r^n,
// p^{n-1}, r^{n-1}, eps, delta (plane x)] (+ [u_p, u_r, g] imaging).
// ADJ = 2: no step; imaging of the coupling C with the forward field whose
// fluxes were just formed: interiors [lam_p, lam_r, delta, g_eps, g_delta]
// ---------------------------------------------------------------------------
template <int M, int ADJ, int GRAD>
struct SUL {
    using B = BX<M>;
    static constexpr bool IMG = ADJ == 2;
    static constexpr int NI = IMG ? 9 : 11 + (GRAD ? 3 : 0);
    static constexpr int OY = 0, OZ = 4 * B::YS, OI = OZ + 4 * B::ZS, SZ = OI + NI * IS;
    static constexpr int HC0 = 0, HCZ = 1, HS0 = 2, HSZ = 3, MM = 4, PC = IMG ? 4 : 5, RC = PC + 1, PP = 7,
                         RP = 8, EP = 9, DE = IMG ? 6 : 10, UP = IMG ? 7 : 11, UR = UP + 1, GG = 13;
    static constexpr uint32_t BYTES = 4u * (4 * B::YR * B::YC + 4 * B::ZR * B::ZC + NI * IS);
};

struct SUMaps {
    CUtensorMap y[4], z[4], h[4], m, pc, rc, pp, rp, e, d, up, ur, g;
};

// x part of pass 2 in push form: the heads hc (centred flux at plane x+M)
// and hs (staggered flux at x+M-1) add their terms to the partial sums of
// planes x .. x+2M (acc[d] is plane x+d):
//   D c at plane i  = sum_k c_k (c_{i+k} - c_{i-k})
//   D- s at plane i = sum_k b_k (s_{i+k-1} - s_{i-k})
template <int M>
WP_DEV void push_x(float2 (&acc)[2 * M + 1], float2 hc, float2 hs, const FDW &w)
{
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const float2 c = f2s(w.c[k - 1]), b = f2s(w.b[k - 1]);
        acc[M - k] = f2fma(c, hc, acc[M - k]);
        acc[M + k] = f2fma(make_float2(-c.x, -c.y), hc, acc[M + k]);
        acc[M - k] = f2fma(b, hs, acc[M - k]);
        acc[M - 1 + k] = f2fma(make_float2(-b.x, -b.y), hs, acc[M - 1 + k]);
    }
}
template <int M>
WP_DEV void shift_x(float2 (&acc)[2 * M + 1])
{
#pragma unroll
    for (int d = 0; d < 2 * M; d++) acc[d] = acc[d + 1];
    acc[2 * M] = make_float2(0.f, 0.f);
}

// y and z parts of sum_i (D_i c_i + D-_i s_i) for one flux pair, both points
template <int M>
WP_DEV float2 yz_part(const float *yc, const float *ys, const float *zc, const float *zs, int iy, int izr, int cz,
                      const FDW &w)
{
    using B = BX<M>;
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const float2 c = f2s(w.c[k - 1]), b = f2s(w.b[k - 1]);
        a = f2fma(c, f2sub(lds2(yc + iy + k * B::YC), lds2(yc + iy - k * B::YC)), a);
        a = f2fma(b, f2sub(lds2(ys + iy + (k - 1) * B::YC), lds2(ys + iy - k * B::YC)), a);
    }
    float wv[2 * M + 2];
    zwin<M>(zc + izr, cz, wv);
#pragma unroll
    for (int k = 1; k <= M; k++)
        a = f2fma(f2s(w.c[k - 1]), make_float2(wv[M + k] - wv[M - k], wv[M + k + 1] - wv[M - k + 1]), a);
    zwin<M>(zs + izr, cz, wv);
#pragma unroll
    for (int k = 1; k <= M; k++)
        a = f2fma(f2s(w.b[k - 1]), make_float2(wv[M + k - 1] - wv[M - k], wv[M + k] - wv[M - k + 1]), a);
    return a;
}

template <int M, int ADJ, int GRAD>
__global__ void __launch_bounds__(NTP, 1)
tti_sp_upd_tma(GridDev g, FDW w, F12 o, const __grid_constant__ SUMaps mp, float *__restrict__ pp,
               float *__restrict__ rp, float *__restrict__ grad, float *__restrict__ zp, float *__restrict__ zr,
               int *flag, int check, int xc, int *err)
{
    using L = SUL<M, ADJ, GRAD>;
    using B = BX<M>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, lane = (ty * TZ2 + tz) & 31;
    const bool lead = ty == 0 && tz == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + 2 * tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        float *I = S + L::OI;
        uint64_t *bar = &bars[st];
        mbar_expect(bar, L::BYTES);
        for (int f = 0; f < 4; f++) {
            tma3(S + L::OY + f * B::YS, &mp.y[f], z0, y0 - M, x, bar);
            tma3(S + L::OZ + f * B::ZS, &mp.z[f], z0 - B::MZ, y0, x, bar);
        }
        tma3(I + L::HC0 * IS, &mp.h[0], z0, y0, x + M, bar);           // beyond NX: zeros
        tma3(I + L::HCZ * IS, &mp.h[1], z0, y0, x + M, bar);
        tma3(I + L::HS0 * IS, &mp.h[2], z0, y0, x + M - 1, bar);
        tma3(I + L::HSZ * IS, &mp.h[3], z0, y0, x + M - 1, bar);
        tma3(I + L::PC * IS, &mp.pc, z0, y0, x, bar);
        tma3(I + L::RC * IS, &mp.rc, z0, y0, x, bar);
        tma3(I + L::DE * IS, &mp.d, z0, y0, x, bar);
        if (L::IMG) {
            tma3(I + L::UP * IS, &mp.up, z0, y0, x, bar);
            tma3(I + L::UR * IS, &mp.ur, z0, y0, x, bar);
            return;
        }
        tma3(I + L::MM * IS, &mp.m, z0, y0, x, bar);
        tma3(I + L::PP * IS, &mp.pp, z0, y0, x, bar);
        tma3(I + L::RP * IS, &mp.rp, z0, y0, x, bar);
        tma3(I + L::EP * IS, &mp.e, z0, y0, x, bar);
        if (GRAD) {
            tma3(I + L::UP * IS, &mp.up, z0, y0, x, bar);
            tma3(I + L::UR * IS, &mp.ur, z0, y0, x, bar);
            tma3(I + L::GG * IS, &mp.g, z0, y0, x, bar);
        }
    };
    Ring R(bars);
    if (lead) {
        R.init();
        ck_begin(g.N, err);
    }
    __syncthreads();
    if (ty >= FY) {                                       // producer warp
        if (lane == 0) R.produce(xa, nit, issue, err);
        return;
    }
    const bool act = y < g.NY && z < g.NZ;
    const unsigned pl = (unsigned)g.NY * (unsigned)g.NZ;
    const unsigned q0 = act ? (unsigned)y * g.NZ + z : 0u;
    const float2 Z2 = make_float2(0.f, 0.f);
    // partial sums of the x terms for planes x .. x+2M: primed with the
    // fluxes of planes xa-M .. xa+M-1 (centred) and xa-M-1 .. xa+M-2
    // (staggered), zero outside the grid
    float2 a0[Q], az[Q];
#pragma unroll
    for (int d = 0; d < Q; d++) a0[d] = az[d] = Z2;
#pragma unroll
    for (int j = 0; j < 2 * M; j++) {
        const int xh = xa - M + j, xs = xh - 1;
        const bool ih_ = act && xh >= 0 && xh < g.NX, is_ = act && xs >= 0 && xs < g.NX;
        push_x<M>(a0, ih_ ? ldg2(o.f[0], xh * pl + q0) : Z2, is_ ? ldg2(o.f[6], xs * pl + q0) : Z2, w);
        push_x<M>(az, ih_ ? ldg2(o.f[3], xh * pl + q0) : Z2, is_ ? ldg2(o.f[9], xs * pl + q0) : Z2, w);
        shift_x<M>(a0);
        shift_x<M>(az);
    }
    const float *sx = g.tab, *sy = g.tab + g.NX, *sz = g.tab + g.NX + g.NY;
    const float dt2 = g.dt * g.dt, hdt = 0.5f * g.dt;
    const float syv = act ? __ldg(sy + y) : 0.f;
    const float syz0 = act ? syv + __ldg(sz + z) : 0.f, syz1 = act ? syv + __ldg(sz + z + 1) : 0.f;
    const int c2 = 2 * tz, ii = ty * FZ + c2;
    const int iy = (ty + M) * B::YC + c2, izr = ty * B::ZC, cz = B::MZ + c2;
    for (int x = xa; x < xb; x++) {
        if (!__all_sync(0xffffffffu, R.wait_full())) {
            if (lane == 0) atomicOr(err, 2);
            return;
        }
        const float *S = sm + R.st * L::SZ;
        const float *I = S + L::OI + ii;
        push_x<M>(a0, lds2(I + L::HC0 * IS), lds2(I + L::HS0 * IS), w);
        push_x<M>(az, lds2(I + L::HCZ * IS), lds2(I + L::HSZ * IS), w);
        if (act) {
            const float *Y = S + L::OY, *Zb = S + L::OZ;
            // flux order in the boxes: c0, cz, s0, sz
            const float2 h0v = f2add(a0[0], yz_part<M>(Y, Y + 2 * B::YS, Zb, Zb + 2 * B::ZS, iy, izr, cz, w));
            const float2 hzv = f2add(az[0], yz_part<M>(Y + B::YS, Y + 3 * B::YS, Zb + B::ZS, Zb + 3 * B::ZS, iy,
                                                       izr, cz, w));
            const unsigned q = x * pl + q0;
            if constexpr (L::IMG) {
                // g_eps += 2 dt^2 lam_p H0 p^n, g_delta += dt^2 (lam_p Hz r^n + lam_r H0 p^n) / sqrt(1 + 2 delta)
                const float2 lp = lds2(I + L::PC * IS), lr = lds2(I + L::RC * IS), d_ = lds2(I + L::DE * IS);
                const float2 ge = lds2(I + L::UP * IS), gd = lds2(I + L::UR * IS);
                const float h0a = h0v.x * g.ih, h0b = h0v.y * g.ih, hza = hzv.x * g.ih, hzb = hzv.y * g.ih;
                st2(grad, q, ge.x + 2.f * dt2 * lp.x * h0a, ge.y + 2.f * dt2 * lp.y * h0b);
                st2(zp, q, gd.x + dt2 * (lp.x * hza + lr.x * h0a) / sqrtf(1.f + 2.f * d_.x),
                    gd.y + dt2 * (lp.y * hzb + lr.y * h0b) / sqrtf(1.f + 2.f * d_.y));
            } else {
                const float2 mm = lds2(I + L::MM * IS), p1 = lds2(I + L::PC * IS), r1 = lds2(I + L::RC * IS);
                const float2 p0 = lds2(I + L::PP * IS), r0 = lds2(I + L::RP * IS);
                const float2 e_ = lds2(I + L::EP * IS), d_ = lds2(I + L::DE * IS);
                const float sxv = __ldg(sx + x);
                const float h0[2] = {h0v.x * g.ih, h0v.y * g.ih}, hz[2] = {hzv.x * g.ih, hzv.y * g.ih};
                const float M2[2] = {mm.x, mm.y}, E2[2] = {e_.x, e_.y}, D2[2] = {d_.x, d_.y};
                const float P1[2] = {p1.x, p1.y}, R1[2] = {r1.x, r1.y}, P0[2] = {p0.x, p0.y}, R0[2] = {r0.x, r0.y};
                const float SYZ[2] = {syz0, syz1};
                float pn[2], rn[2], Lp[2], Lr[2], c1[2], cc[2];
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    c1[i] = 1.f + 2.f * E2[i];
                    cc[i] = sqrtf(1.f + 2.f * D2[i]);
                    Lp[i] = ADJ ? h0[i] : c1[i] * h0[i] + cc[i] * hz[i];
                    Lr[i] = ADJ ? hz[i] : cc[i] * h0[i] + hz[i];
                    const float sd = hdt * (sxv + SYZ[i]);
                    const float A = M2[i] * (1.f + sd), Bc = M2[i] * (1.f - sd);
                    pn[i] = (dt2 * Lp[i] + 2.f * M2[i] * P1[i] - Bc * P0[i]) / A;
                    rn[i] = (dt2 * Lr[i] + 2.f * M2[i] * R1[i] - Bc * R0[i]) / A;
                }
                st2(pp, q, pn[0], pn[1]);
                st2(rp, q, rn[0], rn[1]);
                if (ADJ) {
                    st2(zp, q, c1[0] * pn[0] + cc[0] * rn[0], c1[1] * pn[1] + cc[1] * rn[1]);
                    st2(zr, q, cc[0] * pn[0] + rn[0], cc[1] * pn[1] + rn[1]);
                }
                if (GRAD) {
                    const float2 u = lds2(I + L::UP * IS), v = lds2(I + L::UR * IS), gg = lds2(I + L::GG * IS);
                    st2(grad, q, gg.x - dt2 * (u.x * Lp[0] + v.x * Lr[0]) / M2[0],
                        gg.y - dt2 * (u.y * Lp[1] + v.y * Lr[1]) / M2[1]);
                }
                if (check && !(isfinite(pn[0]) && isfinite(rn[0]) && isfinite(pn[1]) && isfinite(rn[1])))
                    atomicOr(flag, 1);
            }
        }
        shift_x<M>(a0);
        shift_x<M>(az);
        R.release(lane);
    }
}

template <int M, int ADJ, int GRAD>
int sp_launch(prop_s *P, float *const *S, const float *up, const float *ur, float *grad)
{
    using B = BX<M>;
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ2, FY + 2, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    F12 o;                                      // c0_i, cz_i: tmp[0..5]; s0_i, sz_i: tmp[8..13]
    for (int i = 0; i < 6; i++) o.f[i] = t[i];
    for (int i = 0; i < 6; i++) o.f[6 + i] = t[8 + i];
    // pass 1 differentiates (p, r), or zeta = C lam (tmp[6], tmp[7]) in the
    // transposed step
    const float *rp_ = ADJ ? t[6] : S[0], *rr_ = ADJ ? t[7] : S[1];
    SRMaps rm;
    SUMaps um;
    bool ok = map_of(P, rp_, B::RC, B::RR, &rm.p) && map_of(P, rr_, B::RC, B::RR, &rm.r) &&
              map_of(P, rp_, FZ, FY, &rm.qp) && map_of(P, rr_, FZ, FY, &rm.qr) &&
              map_of(P, P->nrm[0], B::PC, B::PR, &rm.nx1) && map_of(P, P->nrm[1], B::PC, B::PR, &rm.ny1) &&
              map_of(P, P->nrm[0], FZ, FY, &rm.nxi);
    // boxes in the order c0, cz, s0, sz; y boxes hold the y fluxes, z boxes
    // the z fluxes, heads the x fluxes
    const int fy[4] = {1, 4, 7, 10}, fz[4] = {2, 5, 8, 11}, fx[4] = {0, 3, 6, 9};
    for (int f = 0; f < 4; f++)
        ok = ok && map_of(P, o.f[fy[f]], B::YC, B::YR, &um.y[f]) && map_of(P, o.f[fz[f]], B::ZC, B::ZR, &um.z[f]) &&
             map_of(P, o.f[fx[f]], FZ, FY, &um.h[f]);
    ok = ok && map_of(P, P->m, FZ, FY, &um.m) && map_of(P, S[0], FZ, FY, &um.pc) &&
         map_of(P, S[1], FZ, FY, &um.rc) && map_of(P, S[2], FZ, FY, &um.pp) && map_of(P, S[3], FZ, FY, &um.rp) &&
         map_of(P, P->eps, FZ, FY, &um.e) && map_of(P, P->del, FZ, FY, &um.d);
    if (GRAD)
        ok = ok && map_of(P, up, FZ, FY, &um.up) && map_of(P, ur, FZ, FY, &um.ur) && map_of(P, grad, FZ, FY, &um.g);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = NSTAGE * SRL<M>::SZ * sizeof(float) + 64, s2 = NSTAGE * SUL<M, ADJ, GRAD>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_sp_rot_tma<M>, s1) && set_smem(tti_sp_upd_tma<M, ADJ, GRAD>, s2);
    (void)attr;
    tti_sp_rot_tma<M><<<grd, blk, s1, P->stream>>>(g, P->w, rp_, rr_, rm, o, xc, P->flag);
    tti_sp_upd_tma<M, ADJ, GRAD><<<grd, blk, s2, P->stream>>>(g, P->w, o, um, S[2], S[3], grad, t[6], t[7], P->flag,
                                                              P->d.check_nan, xc, P->flag);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

template <int M>
int sp_launch_any(prop_s *P, float *const *S, bool adjoint, const float *up, const float *ur, float *grad)
{
    if (!adjoint) return sp_launch<M, 0, 0>(P, S, nullptr, nullptr, nullptr);
    if (!grad) return sp_launch<M, 1, 0>(P, S, nullptr, nullptr, nullptr);
    return sp_launch<M, 1, 1>(P, S, up, ur, grad);
}

// ---------------------------------------------------------------------------
// tilt/azimuth imaging of the staggered-pair operators.  Their bilinear forms
// differ from the centred ones only in the diagonal terms: with a = D zeta_p,
// b = D p, c = D zeta_r, d = D r (centred, at the nodes) and the half-point
// products S0_i(h) = (D+_i zeta_p)(D+_i p)(h), Sz_i(h) = (D+_i zeta_r)(D+_i r)(h),
// the step's term of dJ/dn at node q is the centred one plus
//   2 n_i (T0_i - a_i b_i) - 2 n_i (Tz_i - c_i d_i),
//   T_i(q) = w+ S_i(q) + w- S_i(q - e_i)
// (n(q) enters the two-node averages of the half points q +- 1/2 with weight
// 1/2; at the last node its partner is clamped to itself, weight 1; the
// first node has no half point below it).
// ---------------------------------------------------------------------------
struct SPAxisIn {
    const float *dz[6], *du[6], *s[6], *nx, *ny;
    float *acc[3];
};

__global__ void tti_axis_image_sp(GridDev g, float sc, SPAxisIn a)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= g.N) return;
    const int z = (int)(q % g.NZ), y = (int)((q / g.NZ) % g.NY), x = (int)(q / ((long long)g.NZ * g.NY));
    const int pos[3] = {x, y, z}, len[3] = {g.NX, g.NY, g.NZ};
    const long long str[3] = {(long long)g.NY * g.NZ, g.NZ, 1};
    const float n0 = a.nx[q], n1 = a.ny[q];
    const float nv[3] = {n0, n1, sqrtf(fmaxf(0.f, 1.f - n0 * n0 - n1 * n1))};
    float zp[3], zr[3], gp[3], gr[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        zp[c] = a.dz[c][q];
        zr[c] = a.dz[3 + c][q];
        gp[c] = a.du[c][q];
        gr[c] = a.du[3 + c][q];
    }
    float ng = 0.f, nzp = 0.f, nh = 0.f, nzr = 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        ng += nv[c] * gp[c];
        nzp += nv[c] * zp[c];
        nh += nv[c] * gr[c];
        nzr += nv[c] * zr[c];
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float wp = pos[c] == len[c] - 1 ? 1.f : 0.5f;
        const bool below = pos[c] >= 1;
        const float T0 = wp * a.s[c][q] + (below ? 0.5f * a.s[c][q - str[c]] : 0.f);
        const float Tz = wp * a.s[3 + c][q] + (below ? 0.5f * a.s[3 + c][q - str[c]] : 0.f);
        const float v = zp[c] * ng + nzp * gp[c] - zr[c] * nh - nzr * gr[c] +
                        2.f * nv[c] * ((T0 - zp[c] * gp[c]) - (Tz - zr[c] * gr[c]));
        a.acc[c][q] += sc * v;
    }
}

// eps, delta (and, gax != NULL, tilt/azimuth) imaging of one transposed
// staggered-pair step with the forward field (up, ur) at level n and the
// adjoint field (lp, lr) at level n+1; zeta = C lam in tmp[6], tmp[7].
// Uses tmp[0..5], tmp[8..19].
template <int M>
int sp_image_aniso(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr, float *ge,
                   float *gd, float *const *gax)
{
    using B = BX<M>;
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ2, FY + 2, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    F12 o;
    for (int i = 0; i < 6; i++) o.f[i] = t[i];
    for (int i = 0; i < 6; i++) o.f[6 + i] = t[8 + i];
    SRMaps rm;
    SUMaps um;
    bool ok = map_of(P, up, B::RC, B::RR, &rm.p) && map_of(P, ur, B::RC, B::RR, &rm.r) &&
              map_of(P, up, FZ, FY, &rm.qp) && map_of(P, ur, FZ, FY, &rm.qr) &&
              map_of(P, P->nrm[0], B::PC, B::PR, &rm.nx1) && map_of(P, P->nrm[1], B::PC, B::PR, &rm.ny1) &&
              map_of(P, P->nrm[0], FZ, FY, &rm.nxi);
    const int fy[4] = {1, 4, 7, 10}, fz[4] = {2, 5, 8, 11}, fx[4] = {0, 3, 6, 9};
    for (int f = 0; f < 4; f++)
        ok = ok && map_of(P, o.f[fy[f]], B::YC, B::YR, &um.y[f]) && map_of(P, o.f[fz[f]], B::ZC, B::ZR, &um.z[f]) &&
             map_of(P, o.f[fx[f]], FZ, FY, &um.h[f]);
    ok = ok && map_of(P, lp, FZ, FY, &um.pc) && map_of(P, lr, FZ, FY, &um.rc) && map_of(P, P->del, FZ, FY, &um.d) &&
         map_of(P, ge, FZ, FY, &um.up) && map_of(P, gd, FZ, FY, &um.ur);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = NSTAGE * SRL<M>::SZ * sizeof(float) + 64, s2 = NSTAGE * SUL<M, 2, 0>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_sp_rot_tma<M>, s1) && set_smem(tti_sp_upd_tma<M, 2, 0>, s2);
    (void)attr;
    tti_sp_rot_tma<M><<<grd, blk, s1, P->stream>>>(g, P->w, up, ur, rm, o, xc, P->flag);
    tti_sp_upd_tma<M, 2, 0><<<grd, blk, s2, P->stream>>>(g, P->w, o, um, nullptr, nullptr, ge, gd, nullptr, P->flag,
                                                         0, xc, P->flag);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    if (!gax) return PROP_OK;
    // centred first derivatives of zeta and of the forward field with the
    // staggered half-point products, one rotation pass per pair (zeta_p, u_p)
    // and (zeta_r, u_r), then the pointwise term
    float *dz[6] = {t[0], t[1], t[2], t[3], t[4], t[5]}, *du[6] = {t[8], t[9], t[10], t[11], t[12], t[13]};
    WP_TRY(tti_raw_half_tma(P, t[6], up, dz, du, t + 14));
    WP_TRY(tti_raw_half_tma(P, t[7], ur, dz + 3, du + 3, t + 17));
    const long long n = g.N;
    const unsigned nb = (unsigned)((n + 255) / 256);
    SPAxisIn ai;
    for (int c = 0; c < 6; c++) {
        ai.dz[c] = dz[c];
        ai.du[c] = du[c];
        ai.s[c] = t[14 + c];
    }
    ai.nx = P->nrm[0];
    ai.ny = P->nrm[1];
    for (int c = 0; c < 3; c++) ai.acc[c] = gax[c];
    tti_axis_image_sp<<<nb, 256, 0, P->stream>>>(g, g.dt * g.dt, ai);
    P->kern_launches += 1;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// one staggered-pair TTI step through the TMA-fed passes (same contract as
// tti_sp_launch; NZ a multiple of 4)
int tti_sp_launch_tma(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r, float *grad)
{
    switch (P->M) {
    case 2: return sp_launch_any<2>(P, S, adjoint, img_p, img_r, grad);
    case 4: return sp_launch_any<4>(P, S, adjoint, img_p, img_r, grad);
    case 6: return sp_launch_any<6>(P, S, adjoint, img_p, img_r, grad);
    case 8: return sp_launch_any<8>(P, S, adjoint, img_p, img_r, grad);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

// eps, delta (and tilt/azimuth) imaging of one transposed staggered-pair
// step (see sp_image_aniso; NZ a multiple of 4)
int tti_sp_image_aniso_tma(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr, float *ge,
                           float *gd, float *const *gax)
{
    switch (P->M) {
    case 2: return sp_image_aniso<2>(P, up, ur, lp, lr, ge, gd, gax);
    case 4: return sp_image_aniso<4>(P, up, ur, lp, lr, ge, gd, gax);
    case 6: return sp_image_aniso<6>(P, up, ur, lp, lr, ge, gd, gax);
    case 8: return sp_image_aniso<8>(P, up, ur, lp, lr, ge, gd, gax);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
