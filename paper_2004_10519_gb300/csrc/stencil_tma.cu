// Stencil passes fed by the Tensor Memory Accelerator (sm_103a).
//
// Each CTA owns a 32(z) x FY(y) tile of columns (FY = 8, 16 or 32 rows, one
// compiled set of passes per height, see tma.cuh) and streams along x; each
// of its 16 FY consumer threads updates two adjacent z points, so
// shared-memory taps and global accesses are 8-byte (float2) and every y-tap
// row serves two outputs.  For every plane the y/z-halo boxes of the differentiated fields
// are fetched with cp.async.bulk.tensor into a shared-memory ring of three
// stages (four in the TTI rotation and acoustic forward passes); out-of-grid
// elements arrive as zeros, which is the zero extension of the
// finite-difference operators.  Every other per-plane input (the thread's
// own values, parameters, the new head of each x-derivative queue M planes
// ahead) comes through the same ring as an interior box.  The ring is a
// producer/consumer pipeline on mbarriers (RingN in tma.cuh): a dedicated
// producer warp refills a stage as soon as every consumer warp has released
// it, and no CTA-wide barrier is taken per plane (the acoustic pass uses a
// 32 x 32 tile, two rows per thread).
// z-derivatives read a window of M+1 float2 per field; x-derivatives use
// per-thread float2 register queues.
// Offsets are 32-bit (the runtime keeps N below 2^32).  Every mbarrier wait
// is bounded in time: on expiry the warp sets bit 2 of the error word and
// leaves, the producer first waiting (again bounded) for its copies in
// flight.
//
// Elastic (Sec. IV, Eq. elas1, elastic listing):
//   velocity pass  v <- g (v + dt b_avg Dtau(tau))
//   stress pass    tau <- g (tau + dt C S(v))
// The transposed step is the same two passes with dt -> -dt in the variables
// (b_avg vbar, g C tbar) (the taper, C and the averages are pointwise and
// commute), so adjoint modelling uses these kernels too.
// TTI (Sec. III-A): rotation pass (D of p, r or of zeta = C lam, projected on
// the symmetry axis n) and update pass (divergence, coupling, damped
// leapfrog, fused imaging).  n is read from two precomputed arrays (n_x, n_y
// with n_z >= 0; the operators are quadratic in n, so n and -n agree).
#include "tma.cuh"

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

namespace {

struct F9 {
    float *f[9];
};
struct F5 {
    float *f[5];
};


struct VMaps {
    CUtensorMap xy, yy, xz, zz, yz, b, v[3], qxx, qxy, qxz, bi;
};

// Per consumer thread and tile (32 z x FY y columns at (z0, y0)): position,
// shared-memory offsets and the y/z Cerjan factors of its two z points.
template <int M>
struct ElCtx {
    bool act;
    unsigned q0;             // in-plane offset of the first point
    int cy, cz, c2, ii;      // rows/columns in the halo boxes and the interior box
    int yb1, zb2;            // +1 box row of y+1 and column of z+2 (clamped at the grid end)
    float gzn0, gzh0, gzn1, gzh1, gyn, gyh;
};
template <int M>
WP_DEV ElCtx<M> el_ctx(const GridDev &g, int z0, int y0, int tz, int ty)
{
    using B = BX<M>;
    ElCtx<M> t;
    const int z = z0 + 2 * tz, y = y0 + ty;
    t.act = y < g.NY && z < g.NZ;
    t.q0 = t.act ? (unsigned)y * g.NZ + z : 0u;
    const float *tabz = g.tab + 2 * (g.NX + g.NY);
    const int zc0 = min(z, g.NZ - 1), zc1 = min(z + 1, g.NZ - 1), yc = min(y, g.NY - 1);
    t.gzn0 = __ldg(tabz + 2 * zc0);
    t.gzh0 = __ldg(tabz + 2 * zc0 + 1);
    t.gzn1 = __ldg(tabz + 2 * zc1);
    t.gzh1 = __ldg(tabz + 2 * zc1 + 1);
    t.gyn = __ldg(g.tab + 2 * g.NX + 2 * yc);
    t.gyh = __ldg(g.tab + 2 * g.NX + 2 * yc + 1);
    t.cy = ty + M;
    t.cz = B::MZ + 2 * tz;
    t.c2 = 2 * tz;
    t.ii = ty * FZ + t.c2;
    t.yb1 = y + 1 < g.NY ? ty + 1 : ty;
    t.zb2 = z + 2 < g.NZ ? t.c2 + 2 : t.c2 + 1;
    return t;
}

// ---------------------------------------------------------------------------
// elastic velocity pass, one plane.  ADJ = 1: the velocity half of the
// transposed step in the tbar form, vbar <- g (vbar - dt Dtau(sigma)) with
// sigma = C g tbar in s.f[3..8], and w = b_avg vbar written to o.f[0..2].
// stage: [xy (y box)] [yy (y box)] [xz (z box)] [zz (z box)] [yz (rect)]
//        [b (+1 box)] [v_x v_y v_z (plane x)] [queue heads: xx (x+M),
//        xy (x+M-1), xz (x+M-1)] [b (plane x+1, clamped)]
// x-derivative queues: qxx[j] = t_xx(x - M + 1 + j), qxy[j] = t_xy(x - M + j),
// qxz[j] = t_xz(x - M + j), j = 0 .. 2M-1 (the last entry from the stage).
// ---------------------------------------------------------------------------
template <int M>
struct VL {
    using B = BX<M>;
    static constexpr int OXY = 0, OYY = B::YS, OXZ = 2 * B::YS, OZZ = OXZ + B::ZS, OYZ = OZZ + B::ZS,
                         OB = OYZ + B::RS, OV = OB + B::PS, OQ = OV + 3 * IS, OBX = OQ + 3 * IS,
                         SZ = OBX + IS;
    static constexpr uint32_t BYTES = 4u * (2 * B::YR * B::YC + 2 * B::ZR * B::ZC + B::RR * B::RC +
                                            B::PR * B::PC + 7 * IS);
};

template <int M>
WP_DEV void v_issue(const VMaps &mp, float *S, uint64_t *bar, int z0, int y0, int x, int NX)
{
    using L = VL<M>;
    using B = BX<M>;
    mbar_expect(bar, L::BYTES);
    tma3(S + L::OXY, &mp.xy, z0, y0 - M, x, bar);
    tma3(S + L::OYY, &mp.yy, z0, y0 - M, x, bar);
    tma3(S + L::OXZ, &mp.xz, z0 - B::MZ, y0, x, bar);
    tma3(S + L::OZZ, &mp.zz, z0 - B::MZ, y0, x, bar);
    tma3(S + L::OYZ, &mp.yz, z0 - B::MZ, y0 - M, x, bar);
    tma3(S + L::OB, &mp.b, z0, y0, x, bar);
    for (int i = 0; i < 3; i++) tma3(S + L::OV + i * IS, &mp.v[i], z0, y0, x, bar);
    tma3(S + L::OQ, &mp.qxx, z0, y0, x + M, bar);                  // beyond NX: zeros
    tma3(S + L::OQ + IS, &mp.qxy, z0, y0, x + M - 1, bar);
    tma3(S + L::OQ + 2 * IS, &mp.qxz, z0, y0, x + M - 1, bar);
    tma3(S + L::OBX, &mp.bi, z0, y0, min(x + 1, NX - 1), bar);
}

template <int M>
WP_DEV void v_preload(const GridDev &g, const F9 &s, const ElCtx<M> &t, int xa, float2 (&qxx)[2 * M],
                      float2 (&qxy)[2 * M], float2 (&qxz)[2 * M])
{
    const unsigned pl = (unsigned)g.NY * (unsigned)g.NZ;
    const float2 Z2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 2 * M - 1; j++) {
        const int xq = xa - M + 1 + j, xr = xa - M + j;
        qxx[j] = t.act && xq >= 0 && xq < g.NX ? ldg2(s.f[3], xq * pl + t.q0) : Z2;
        qxy[j] = t.act && xr >= 0 && xr < g.NX ? ldg2(s.f[6], xr * pl + t.q0) : Z2;
        qxz[j] = t.act && xr >= 0 && xr < g.NX ? ldg2(s.f[7], xr * pl + t.q0) : Z2;
    }
}

template <int M, int ADJ>
WP_DEV void v_plane(const GridDev &g, const FDW &w, const F9 &s, const F5 &o, const float *S, const ElCtx<M> &t,
                    int x, float2 (&qxx)[2 * M], float2 (&qxy)[2 * M], float2 (&qxz)[2 * M])
{
    using L = VL<M>;
    using B = BX<M>;
    constexpr int Q = 2 * M;
    const float2 Z2 = make_float2(0.f, 0.f);
    qxx[Q - 1] = lds2(S + L::OQ + t.ii);
    qxy[Q - 1] = lds2(S + L::OQ + IS + t.ii);
    qxz[Q - 1] = lds2(S + L::OQ + 2 * IS + t.ii);
    if (t.act) {
        const int cy = t.cy, cz = t.cz, c2 = t.c2, ii = t.ii;
        const float c = g.dt * g.ih;
        const float *sxy = S + L::OXY, *syy = S + L::OYY, *syz = S + L::OYZ, *sb = S + L::OB;
        float wxz[2 * M + 2], wyz[2 * M + 2], wzz[2 * M + 2];
        zwin<M>(S + L::OXZ + (cy - M) * B::ZC, cz, wxz);
        zwin<M>(syz + cy * B::RC, cz, wyz);
        zwin<M>(S + L::OZZ + (cy - M) * B::ZC, cz, wzz);
        float2 d0 = Z2, d1 = Z2, d2 = Z2;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const float2 b = f2s(w.b[k - 1]);
            const float2 ax = f2sub(qxx[M - 1 + k], qxx[M - k]);
            const float2 ay = f2sub(lds2(sxy + (cy + k - 1) * B::YC + c2), lds2(sxy + (cy - k) * B::YC + c2));
            const float2 az = make_float2(wxz[M + k - 1] - wxz[M - k], wxz[M + k] - wxz[M - k + 1]);
            d0 = f2fma(b, f2add(f2add(ax, ay), az), d0);
            const float2 bx_ = f2sub(qxy[M + k - 1], qxy[M - k]);
            const float2 by_ = f2sub(lds2(syy + (cy + k) * B::YC + c2), lds2(syy + (cy - k + 1) * B::YC + c2));
            const float2 bz_ = make_float2(wyz[M + k - 1] - wyz[M - k], wyz[M + k] - wyz[M - k + 1]);
            d1 = f2fma(b, f2add(f2add(bx_, by_), bz_), d1);
            const float2 cx_ = f2sub(qxz[M + k - 1], qxz[M - k]);
            const float2 cy_ = f2sub(lds2(syz + (cy + k - 1) * B::RC + cz), lds2(syz + (cy - k) * B::RC + cz));
            const float2 cz_ = make_float2(wzz[M + k] - wzz[M - k + 1], wzz[M + k + 1] - wzz[M - k + 2]);
            d2 = f2fma(b, f2add(f2add(cx_, cy_), cz_), d2);
        }
        const float d0a = d0.x, d0b = d0.y, d1a = d1.x, d1b = d1.y, d2a = d2.x, d2b = d2.y;
        const float2 v0 = lds2(S + L::OV + ii), v1 = lds2(S + L::OV + IS + ii), v2 = lds2(S + L::OV + 2 * IS + ii);
        const float2 bxn = lds2(S + L::OBX + ii);
        const int ty = cy - M;
        const float2 b0 = lds2(sb + ty * B::PC + c2);
        const float2 bY = lds2(sb + t.yb1 * B::PC + c2);
        const float bz2 = sb[ty * B::PC + t.zb2];
        const float gxn = __ldg(g.tab + 2 * x), gxh = __ldg(g.tab + 2 * x + 1);
        const unsigned q = x * (unsigned)g.NY * (unsigned)g.NZ + t.q0;
        // face averages of buoyancy and tapers at the three velocity points
        const float bxa = 0.5f * (b0.x + bxn.x), bxb = 0.5f * (b0.y + bxn.y);
        const float bya = 0.5f * (b0.x + bY.x), byb = 0.5f * (b0.y + bY.y);
        const float bza = 0.5f * (b0.x + b0.y), bzb = 0.5f * (b0.y + bz2);
        const float gx0 = gxh * t.gyn * t.gzn0, gx1 = gxh * t.gyn * t.gzn1;
        const float gy0 = gxn * t.gyh * t.gzn0, gy1 = gxn * t.gyh * t.gzn1;
        const float gz0 = gxn * t.gyn * t.gzh0, gz1 = gxn * t.gyn * t.gzh1;
        if (!ADJ) {
            st2(s.f[0], q, gx0 * (v0.x + c * bxa * d0a), gx1 * (v0.y + c * bxb * d0b));
            st2(s.f[1], q, gy0 * (v1.x + c * bya * d1a), gy1 * (v1.y + c * byb * d1b));
            st2(s.f[2], q, gz0 * (v2.x + c * bza * d2a), gz1 * (v2.y + c * bzb * d2b));
        } else {
            const float u0a = gx0 * (v0.x - c * d0a), u0b = gx1 * (v0.y - c * d0b);
            const float u1a = gy0 * (v1.x - c * d1a), u1b = gy1 * (v1.y - c * d1b);
            const float u2a = gz0 * (v2.x - c * d2a), u2b = gz1 * (v2.y - c * d2b);
            st2(s.f[0], q, u0a, u0b);
            st2(s.f[1], q, u1a, u1b);
            st2(s.f[2], q, u2a, u2b);
            st2(o.f[0], q, bxa * u0a, bxb * u0b);
            st2(o.f[1], q, bya * u1a, byb * u1b);
            st2(o.f[2], q, bza * u2a, bzb * u2b);
        }
    }
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qxx[j] = qxx[j + 1];
        qxy[j] = qxy[j + 1];
        qxz[j] = qxz[j + 1];
    }
}

// one tile (bx, by: z and y tile; bz: x chunk of xc planes)
template <int M, int ADJ>
WP_DEV void el_vpass_body(const GridDev &g, const FDW &w, const F9 &s, const F5 &o, const VMaps &mp, int bx,
                          int by, int bz, int xc, int *err)
{
    using L = VL<M>;
    constexpr int Q = 2 * M;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, warp = (ty * TZ2 + tz) >> 5, lane = (ty * TZ2 + tz) & 31;
    const bool lead = warp == 0 && lane == 0;
    const int z0 = bx * FZ, y0 = by * FY;
    const int xa = bz * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) { v_issue<M>(mp, sm + st * L::SZ, &bars[st], z0, y0, x, g.NX); };
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
    const ElCtx<M> t = el_ctx<M>(g, z0, y0, tz, ty);
    float2 qxx[Q], qxy[Q], qxz[Q];
    v_preload<M>(g, s, t, xa, qxx, qxy, qxz);
    for (int x = xa; x < xb; x++) {
        if (!__all_sync(0xffffffffu, R.wait_full())) {
            if (lane == 0) atomicOr(err, 2);
            return;
        }
        v_plane<M, ADJ>(g, w, s, o, sm + R.st * L::SZ, t, x, qxx, qxy, qxz);
        R.release(lane);
    }
}

template <int M, int ADJ>
__global__ void __launch_bounds__(NTP, occ(M <= 4 ? 2 : 1))
el_vpass_tma(GridDev g, FDW w, F9 s, F5 o, const __grid_constant__ VMaps mp, int xc, int *err)
{
    el_vpass_body<M, ADJ>(g, w, s, o, mp, blockIdx.x, blockIdx.y, blockIdx.z, xc, err);
}

// ---------------------------------------------------------------------------
// elastic stress pass, one plane: the strain S(v) of a velocity triple
// (s.f[0..2]) and
//   MODE 0  tau <- g (tau + dt C S(v))                     (forward step)
//   MODE 1  tbar <- t - dt S(w), t = g tbar, w = b_avg vbar  (stress half of
//           the transposed step in the tbar form; t read, tbar written in
//           s.f[3..8])
//   MODE 2  imaging with the forward v^{k+1}: g_lambda += dt tr(t) tr(S v),
//           g_mu += 2 dt sum_i t_ii S_ii, edge products dt t_c S_c
//           (o.f = g_lambda, g_mu, xy, xz, yz products)
// stage: [vx rect] [vy rect] [vz rect] (+ [mu +1 box, planes x, x+1] MODE 0)
//        [t_xx .. t_yz (plane x)] (+ [lambda] MODE 0) (+ [g_lambda, g_mu]
//        MODE 2) [queue heads: vx (x+M-1), vy (x+M), vz (x+M)]
// x-derivative queues: qvx[j] = v_x(x - M + j), qvy[j] = v_y(x - M + 1 + j),
// qvz[j] = v_z(x - M + 1 + j).
// ---------------------------------------------------------------------------
template <int M, int MODE>
struct TL {
    using B = BX<M>;
    static constexpr int NP = MODE == 0 ? 2 : 0;           // +1 boxes
    static constexpr int NI = 6 + (MODE == 0 ? 1 : 0) + (MODE == 2 ? 2 : 0) + 3;
    static constexpr int OVX = 0, OVY = B::RS, OVZ = 2 * B::RS, OM0 = 3 * B::RS, OM1 = OM0 + B::PS,
                         OT = 3 * B::RS + NP * B::PS, OL = OT + 6 * IS, OG = OL + (MODE == 0 ? IS : 0),
                         OQ = OG + (MODE == 2 ? 2 * IS : 0), SZ = OQ + 3 * IS;
    static constexpr uint32_t BYTES = 4u * (3 * B::RR * B::RC + NP * B::PR * B::PC + NI * IS);
};

struct TMaps {
    CUtensorMap vx, vy, vz, mu, t[6], lam, qvx, qvy, qvz, gl, gm;
};

template <int M, int MODE>
WP_DEV void t_issue(const TMaps &mp, float *S, uint64_t *bar, int z0, int y0, int x, int NX)
{
    using L = TL<M, MODE>;
    using B = BX<M>;
    mbar_expect(bar, L::BYTES);
    tma3(S + L::OVX, &mp.vx, z0 - B::MZ, y0 - M, x, bar);
    tma3(S + L::OVY, &mp.vy, z0 - B::MZ, y0 - M, x, bar);
    tma3(S + L::OVZ, &mp.vz, z0 - B::MZ, y0 - M, x, bar);
    if (MODE == 0) {
        tma3(S + L::OM0, &mp.mu, z0, y0, x, bar);
        tma3(S + L::OM1, &mp.mu, z0, y0, min(x + 1, NX - 1), bar);
        tma3(S + L::OL, &mp.lam, z0, y0, x, bar);
    }
    for (int i = 0; i < 6; i++) tma3(S + L::OT + i * IS, &mp.t[i], z0, y0, x, bar);
    if (MODE == 2) {
        tma3(S + L::OG, &mp.gl, z0, y0, x, bar);
        tma3(S + L::OG + IS, &mp.gm, z0, y0, x, bar);
    }
    tma3(S + L::OQ, &mp.qvx, z0, y0, x + M - 1, bar);              // beyond NX: zeros
    tma3(S + L::OQ + IS, &mp.qvy, z0, y0, x + M, bar);
    tma3(S + L::OQ + 2 * IS, &mp.qvz, z0, y0, x + M, bar);
}

template <int M>
WP_DEV void t_preload(const GridDev &g, const F9 &s, const ElCtx<M> &t, int xa, float2 (&qvx)[2 * M],
                      float2 (&qvy)[2 * M], float2 (&qvz)[2 * M])
{
    const unsigned pl = (unsigned)g.NY * (unsigned)g.NZ;
    const float2 Z2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 2 * M - 1; j++) {
        const int xr = xa - M + j, xq = xa - M + 1 + j;
        qvx[j] = t.act && xr >= 0 && xr < g.NX ? ldg2(s.f[0], xr * pl + t.q0) : Z2;
        qvy[j] = t.act && xq >= 0 && xq < g.NX ? ldg2(s.f[1], xq * pl + t.q0) : Z2;
        qvz[j] = t.act && xq >= 0 && xq < g.NX ? ldg2(s.f[2], xq * pl + t.q0) : Z2;
    }
}

template <int M, int MODE>
WP_DEV void t_plane(const GridDev &g, const FDW &w, const F9 &s, const F5 &o, const float *S, const ElCtx<M> &t,
                    int x, float2 (&qvx)[2 * M], float2 (&qvy)[2 * M], float2 (&qvz)[2 * M])
{
    using L = TL<M, MODE>;
    using B = BX<M>;
    constexpr int Q = 2 * M;
    const float2 Z2 = make_float2(0.f, 0.f);
    qvx[Q - 1] = lds2(S + L::OQ + t.ii);
    qvy[Q - 1] = lds2(S + L::OQ + IS + t.ii);
    qvz[Q - 1] = lds2(S + L::OQ + 2 * IS + t.ii);
    if (t.act) {
        const int cy = t.cy, cz = t.cz, c2 = t.c2, ii = t.ii, ty = t.cy - M;
        const float c = g.dt * g.ih;
        const float *svx = S + L::OVX, *svy = S + L::OVY, *svz = S + L::OVZ;
        float wvx[2 * M + 2], wvy[2 * M + 2], wvz[2 * M + 2];
        zwin<M>(svx + cy * B::RC, cz, wvx);
        zwin<M>(svy + cy * B::RC, cz, wvy);
        zwin<M>(svz + cy * B::RC, cz, wvz);
        float2 ex = Z2, ey = Z2, ez = Z2, gxy = Z2, gxz = Z2, gyz = Z2;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const float2 b = f2s(w.b[k - 1]);
            ex = f2fma(b, f2sub(qvx[M + k - 1], qvx[M - k]), ex);
            ey = f2fma(b, f2sub(lds2(svy + (cy + k - 1) * B::RC + cz), lds2(svy + (cy - k) * B::RC + cz)), ey);
            ez = f2fma(b, make_float2(wvz[M + k - 1] - wvz[M - k], wvz[M + k] - wvz[M - k + 1]), ez);
            const float2 xy = f2sub(lds2(svx + (cy + k) * B::RC + cz), lds2(svx + (cy - k + 1) * B::RC + cz));
            const float2 yx = f2sub(qvy[M - 1 + k], qvy[M - k]);
            gxy = f2fma(b, f2add(xy, yx), gxy);
            const float2 zx = f2sub(qvz[M - 1 + k], qvz[M - k]);
            const float2 xz = make_float2(wvx[M + k] - wvx[M - k + 1], wvx[M + k + 1] - wvx[M - k + 2]);
            gxz = f2fma(b, f2add(xz, zx), gxz);
            const float2 zy = f2sub(lds2(svz + (cy + k) * B::RC + cz), lds2(svz + (cy - k + 1) * B::RC + cz));
            const float2 yz = make_float2(wvy[M + k] - wvy[M - k + 1], wvy[M + k + 1] - wvy[M - k + 2]);
            gyz = f2fma(b, f2add(yz, zy), gyz);
        }
        const float exa = ex.x, exb = ex.y, eya = ey.x, eyb = ey.y, eza = ez.x, ezb = ez.y;
        const float gxya = gxy.x, gxyb = gxy.y, gxza = gxz.x, gxzb = gxz.y, gyza = gyz.x, gyzb = gyz.y;
        const float *T = S + L::OT + ii;
        const float2 t0 = lds2(T), t1 = lds2(T + IS), t2 = lds2(T + 2 * IS);
        const float2 t3 = lds2(T + 3 * IS), t4 = lds2(T + 4 * IS), t5 = lds2(T + 5 * IS);
        const unsigned q = x * (unsigned)g.NY * (unsigned)g.NZ + t.q0;
        if (MODE == 0) {
            const float *R0 = S + L::OM0, *R1 = S + L::OM1;
            const float2 m0 = lds2(R0 + ty * B::PC + c2), my = lds2(R0 + t.yb1 * B::PC + c2);
            const float2 mx = lds2(R1 + ty * B::PC + c2), mxy_ = lds2(R1 + t.yb1 * B::PC + c2);
            const float m0z = R0[ty * B::PC + t.zb2], myz = R0[t.yb1 * B::PC + t.zb2], mxz = R1[ty * B::PC + t.zb2];
            const float2 l = lds2(S + L::OL + ii);
            const float gxn = __ldg(g.tab + 2 * x), gxh = __ldg(g.tab + 2 * x + 1);
            const float gyn = t.gyn, gyh = t.gyh, gzn0 = t.gzn0, gzn1 = t.gzn1, gzh0 = t.gzh0, gzh1 = t.gzh1;
            const float gn0 = gxn * gyn * gzn0, gn1 = gxn * gyn * gzn1;
            // averages of mu over the 4 nodes around each edge (the pair's
            // second lane is the first point's z+1 neighbour)
            const float mxya = 0.25f * (m0.x + mx.x + my.x + mxy_.x);
            const float mxza = 0.25f * (m0.x + mx.x + m0.y + mx.y);
            const float myza = 0.25f * (m0.x + my.x + m0.y + my.y);
            const float mxyb = 0.25f * (m0.y + mx.y + my.y + mxy_.y);
            const float mxzb = 0.25f * (m0.y + mx.y + m0z + mxz);
            const float myzb = 0.25f * (m0.y + my.y + m0z + myz);
            const float tra = exa + eya + eza, trb = exb + eyb + ezb;
            const float m2a = 2.f * m0.x, m2b = 2.f * m0.y;
            st2(s.f[3], q, gn0 * (t0.x + c * (l.x * tra + m2a * exa)), gn1 * (t0.y + c * (l.y * trb + m2b * exb)));
            st2(s.f[4], q, gn0 * (t1.x + c * (l.x * tra + m2a * eya)), gn1 * (t1.y + c * (l.y * trb + m2b * eyb)));
            st2(s.f[5], q, gn0 * (t2.x + c * (l.x * tra + m2a * eza)), gn1 * (t2.y + c * (l.y * trb + m2b * ezb)));
            st2(s.f[6], q, gxh * gyh * gzn0 * (t3.x + c * mxya * gxya), gxh * gyh * gzn1 * (t3.y + c * mxyb * gxyb));
            st2(s.f[7], q, gxh * gyn * gzh0 * (t4.x + c * mxza * gxza), gxh * gyn * gzh1 * (t4.y + c * mxzb * gxzb));
            st2(s.f[8], q, gxn * gyh * gzh0 * (t5.x + c * myza * gyza), gxn * gyh * gzh1 * (t5.y + c * myzb * gyzb));
        } else if (MODE == 1) {
            st2(s.f[3], q, t0.x - c * exa, t0.y - c * exb);
            st2(s.f[4], q, t1.x - c * eya, t1.y - c * eyb);
            st2(s.f[5], q, t2.x - c * eza, t2.y - c * ezb);
            st2(s.f[6], q, t3.x - c * gxya, t3.y - c * gxyb);
            st2(s.f[7], q, t4.x - c * gxza, t4.y - c * gxzb);
            st2(s.f[8], q, t5.x - c * gyza, t5.y - c * gyzb);
        } else {
            const float2 gl = lds2(S + L::OG + ii), gm = lds2(S + L::OG + IS + ii);
            st2(o.f[0], q, gl.x + c * (t0.x + t1.x + t2.x) * (exa + eya + eza),
                gl.y + c * (t0.y + t1.y + t2.y) * (exb + eyb + ezb));
            st2(o.f[1], q, gm.x + 2.f * c * (t0.x * exa + t1.x * eya + t2.x * eza),
                gm.y + 2.f * c * (t0.y * exb + t1.y * eyb + t2.y * ezb));
            // edge products summed over the steps (gathered onto the nodes at the end)
            const float2 p3 = *reinterpret_cast<const float2 *>(o.f[2] + q);
            const float2 p4 = *reinterpret_cast<const float2 *>(o.f[3] + q);
            const float2 p5 = *reinterpret_cast<const float2 *>(o.f[4] + q);
            st2(o.f[2], q, p3.x + c * t3.x * gxya, p3.y + c * t3.y * gxyb);
            st2(o.f[3], q, p4.x + c * t4.x * gxza, p4.y + c * t4.y * gxzb);
            st2(o.f[4], q, p5.x + c * t5.x * gyza, p5.y + c * t5.y * gyzb);
        }
    }
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qvx[j] = qvx[j + 1];
        qvy[j] = qvy[j + 1];
        qvz[j] = qvz[j + 1];
    }
}

template <int M, int MODE>
WP_DEV void el_tpass_body(const GridDev &g, const FDW &w, const F9 &s, const F5 &o, const TMaps &mp, int bx,
                          int by, int bz, int xc, int *err)
{
    using L = TL<M, MODE>;
    constexpr int Q = 2 * M;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, warp = (ty * TZ2 + tz) >> 5, lane = (ty * TZ2 + tz) & 31;
    const bool lead = warp == 0 && lane == 0;
    const int z0 = bx * FZ, y0 = by * FY;
    const int xa = bz * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) { t_issue<M, MODE>(mp, sm + st * L::SZ, &bars[st], z0, y0, x, g.NX); };
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
    const ElCtx<M> t = el_ctx<M>(g, z0, y0, tz, ty);
    float2 qvx[Q], qvy[Q], qvz[Q];
    t_preload<M>(g, s, t, xa, qvx, qvy, qvz);
    for (int x = xa; x < xb; x++) {
        if (!__all_sync(0xffffffffu, R.wait_full())) {
            if (lane == 0) atomicOr(err, 2);
            return;
        }
        t_plane<M, MODE>(g, w, s, o, sm + R.st * L::SZ, t, x, qvx, qvy, qvz);
        R.release(lane);
    }
}

template <int M, int MODE>
__global__ void __launch_bounds__(NTP, occ(M <= 4 ? 2 : 1))
el_tpass_tma(GridDev g, FDW w, F9 s, F5 o, const __grid_constant__ TMaps mp, int xc, int *err)
{
    el_tpass_body<M, MODE>(g, w, s, o, mp, blockIdx.x, blockIdx.y, blockIdx.z, xc, err);
}

// batched elastic passes: per-shot entries (grid with the step's dt,
// fields, maps) and a tile table over all shots, as for TTI
struct ElShot {
    VMaps vm;
    TMaps tm;
    GridDev g;
    F9 s;
    F5 o;
    int xc;
    int *flag;
};

template <int M, int ADJ>
__global__ void __launch_bounds__(NTP, occ(M <= 4 ? 2 : 1))
el_vpass_batch(const ElShot *__restrict__ shots, const int4 *__restrict__ tiles, FDW w)
{
    const int4 tl = tiles[blockIdx.x];
    const ElShot &S = shots[tl.x];
    el_vpass_body<M, ADJ>(S.g, w, S.s, S.o, S.vm, tl.y, tl.z, tl.w, S.xc, S.flag);
}

template <int M, int MODE>
__global__ void __launch_bounds__(NTP, occ(M <= 4 ? 2 : 1))
el_tpass_batch(const ElShot *__restrict__ shots, const int4 *__restrict__ tiles, FDW w)
{
    const int4 tl = tiles[blockIdx.x];
    const ElShot &S = shots[tl.x];
    el_tpass_body<M, MODE>(S.g, w, S.s, S.o, S.tm, tl.y, tl.z, tl.w, S.xc, S.flag);
}

// ---------------------------------------------------------------------------
// TTI rotation pass on (p, r), or on zeta = C lam in the transposed step
// (the update pass of the previous adjoint step writes zeta).  MODE 1: write
// the unprojected first derivatives D p, D r (tilt/azimuth imaging).  MODE 2:
// also the products of the staggered first derivatives at the half points,
// h_i = (D+_i p)(D+_i r), D+_i f(q + 1/2) = sum_k b_k (f(q + k e_i) -
// f(q - (k - 1) e_i)) / h, zero outside the grid (staggered-pair tilt/azimuth
// imaging with p = zeta_p, r = u_p or p = zeta_r, r = u_r)
// stage: [p rect] [r rect] [queue heads p, r (x+M)] [n_x, n_y (plane x)]
// ---------------------------------------------------------------------------
template <int M>
struct RL {
    using B = BX<M>;
    static constexpr int OP = 0, OR = B::RS, OQ = 2 * B::RS, ON = OQ + 2 * IS, SZ = ON + 2 * IS;
    static constexpr uint32_t BYTES = 4u * (2 * B::RR * B::RC + 4 * IS);
    static constexpr int NS = 4;         // ring stages (two CTAs per SM still fit)
};

struct RMaps {
    CUtensorMap p, r, qp, qr, nx, ny;
};

// one tile (bx, by: 32 z x FY y columns; bz: x chunk of xc planes)
struct F3 {
    float *f[3];
};

template <int M, int MODE>
WP_DEV void tti_rot_body(const GridDev &g, const FDW &w, const float *__restrict__ p,
                         const float *__restrict__ r, const RMaps &mp, float *__restrict__ ex,
                         float *__restrict__ ey, float *__restrict__ ez, float *__restrict__ fx,
                         float *__restrict__ fy, float *__restrict__ fz, const F3 &hh, int bx, int by, int bz,
                         int xc, int *err)
{
    constexpr bool RAW = MODE != 0, HALF = MODE == 2;
    using L = RL<M>;
    using B = BX<M>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::NS * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, lane = (ty * TZ2 + tz) & 31;
    const bool lead = ty == 0 && tz == 0;
    const int z0 = bx * FZ, y0 = by * FY;
    const int z = z0 + 2 * tz, y = y0 + ty;
    const int xa = bz * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        uint64_t *bar = &bars[st];
        mbar_expect(bar, L::BYTES);
        tma3(S + L::OP, &mp.p, z0 - B::MZ, y0 - M, x, bar);
        tma3(S + L::OR, &mp.r, z0 - B::MZ, y0 - M, x, bar);
        tma3(S + L::OQ, &mp.qp, z0, y0, x + M, bar);                  // beyond NX: zeros
        tma3(S + L::OQ + IS, &mp.qr, z0, y0, x + M, bar);
        tma3(S + L::ON, &mp.nx, z0, y0, x, bar);
        tma3(S + L::ON + IS, &mp.ny, z0, y0, x, bar);
    };
    RingN<L::NS> R(bars);
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
    const int cy = ty + M, cz = B::MZ + 2 * tz, ii = ty * FZ + 2 * tz;
    const int ci = cy * B::RC + cz;
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
            float wp[2 * M + 2], wr[2 * M + 2];
            zwin<M>(sp + cy * B::RC, cz, wp);
            zwin<M>(sr + cy * B::RC, cz, wr);
            // paired FP32: .x the first z point, .y the second
            float2 gp0 = Z2, gp1 = Z2, gp2 = Z2, gr0 = Z2, gr1 = Z2, gr2 = Z2;
            float2 hp0 = Z2, hp1 = Z2, hp2 = Z2, hr0 = Z2, hr1 = Z2, hr2 = Z2;   // HALF: staggered sums
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float2 c = f2s(w.c[k - 1]);
                gp0 = f2fma(c, f2sub(qp[M + k], qp[M - k]), gp0);
                gr0 = f2fma(c, f2sub(qr[M + k], qr[M - k]), gr0);
                gp1 = f2fma(c, f2sub(lds2(sp + ci + k * B::RC), lds2(sp + ci - k * B::RC)), gp1);
                gr1 = f2fma(c, f2sub(lds2(sr + ci + k * B::RC), lds2(sr + ci - k * B::RC)), gr1);
                gp2 = f2fma(c, make_float2(wp[M + k] - wp[M - k], wp[M + k + 1] - wp[M - k + 1]), gp2);
                gr2 = f2fma(c, make_float2(wr[M + k] - wr[M - k], wr[M + k + 1] - wr[M - k + 1]), gr2);
                if constexpr (HALF) {
                    const float2 b = f2s(w.b[k - 1]);
                    hp0 = f2fma(b, f2sub(qp[M + k], qp[M - k + 1]), hp0);
                    hr0 = f2fma(b, f2sub(qr[M + k], qr[M - k + 1]), hr0);
                    hp1 = f2fma(b, f2sub(lds2(sp + ci + k * B::RC), lds2(sp + ci - (k - 1) * B::RC)), hp1);
                    hr1 = f2fma(b, f2sub(lds2(sr + ci + k * B::RC), lds2(sr + ci - (k - 1) * B::RC)), hr1);
                    hp2 = f2fma(b, make_float2(wp[M + k] - wp[M - k + 1], wp[M + k + 1] - wp[M - k + 2]), hp2);
                    hr2 = f2fma(b, make_float2(wr[M + k] - wr[M - k + 1], wr[M + k + 1] - wr[M - k + 2]), hr2);
                }
            }
            const float gp0a = gp0.x, gp0b = gp0.y, gp1a = gp1.x, gp1b = gp1.y, gp2a = gp2.x, gp2b = gp2.y;
            const float gr0a = gr0.x, gr0b = gr0.y, gr1a = gr1.x, gr1b = gr1.y, gr2a = gr2.x, gr2b = gr2.y;
            const float2 n0 = lds2(S + L::ON + ii), n1 = lds2(S + L::ON + IS + ii);
            const float ih = g.ih;
            const unsigned q = x * pl + q0;
            const float gp[2][3] = {{gp0a * ih, gp1a * ih, gp2a * ih}, {gp0b * ih, gp1b * ih, gp2b * ih}};
            const float gr[2][3] = {{gr0a * ih, gr1a * ih, gr2a * ih}, {gr0b * ih, gr1b * ih, gr2b * ih}};
            const float nx2[2] = {n0.x, n0.y}, ny2[2] = {n1.x, n1.y};
            float o[2][6];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                if constexpr (RAW) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        o[i][c] = gp[i][c];
                        o[i][3 + c] = gr[i][c];
                    }
                    continue;
                }
                const float a0 = nx2[i], a1 = ny2[i];
                const float a2 = sqrtf(fmaxf(0.f, 1.f - a0 * a0 - a1 * a1));
                const float wpn = a0 * gp[i][0] + a1 * gp[i][1] + a2 * gp[i][2];
                const float wrn = a0 * gr[i][0] + a1 * gr[i][1] + a2 * gr[i][2];
                o[i][0] = gp[i][0] - a0 * wpn;
                o[i][1] = gp[i][1] - a1 * wpn;
                o[i][2] = gp[i][2] - a2 * wpn;
                o[i][3] = a0 * wrn;
                o[i][4] = a1 * wrn;
                o[i][5] = a2 * wrn;
            }
            st2(ex, q, o[0][0], o[1][0]);
            st2(ey, q, o[0][1], o[1][1]);
            st2(ez, q, o[0][2], o[1][2]);
            st2(fx, q, o[0][3], o[1][3]);
            st2(fy, q, o[0][4], o[1][4]);
            st2(fz, q, o[0][5], o[1][5]);
            if constexpr (HALF) {
                const float ih2 = ih * ih;
                st2(hh.f[0], q, hp0.x * hr0.x * ih2, hp0.y * hr0.y * ih2);
                st2(hh.f[1], q, hp1.x * hr1.x * ih2, hp1.y * hr1.y * ih2);
                st2(hh.f[2], q, hp2.x * hr2.x * ih2, hp2.y * hr2.y * ih2);
            }
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qp[j] = qp[j + 1];
            qr[j] = qr[j + 1];
        }
        R.release(lane);
    }
}

template <int M, int MODE = 0>
__global__ void __launch_bounds__(NTP, occ(MODE == 2 && M > 6 ? 1 : 2))
tti_rot_tma(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
            const __grid_constant__ RMaps mp, float *__restrict__ ex, float *__restrict__ ey,
            float *__restrict__ ez, float *__restrict__ fx, float *__restrict__ fy, float *__restrict__ fz,
            F3 hh, int xc, int *err)
{
    tti_rot_body<M, MODE>(g, w, p, r, mp, ex, ey, ez, fx, fy, fz, hh, blockIdx.x, blockIdx.y, blockIdx.z, xc,
                          err);
}

// ---------------------------------------------------------------------------
// TTI update pass.  ADJ = 1: the transposed step, which also writes
// zeta = C lam of the new level (zp, zr) for the next rotation pass.
// ADJ = 2: no step; imaging of the coupling C with the forward field whose
// rotated intermediates were just formed: with h = [H0 p^n; Hz r^n] and
// lam = lam^{n+1} (pc, rc), g_eps (grad) += 2 dt^2 lam_p H0 p^n and
// g_delta (zp) += dt^2 (lam_p Hz r^n + lam_r H0 p^n) / sqrt(1 + 2 delta)
// (dC/deps = [[2, 0], [0, 0]], dC/ddelta = [[0, s'], [s', 0]]).
// stage: [e_y y box] [f_y y box] [e_z z box] [f_z z box] [queue heads e_x,
//        f_x (x+M)] [m, p^n, r^n, p^{n-1}, r^{n-1}, eps, del (plane x)]
//        (+ [u_p, u_r, g] imaging)
// ---------------------------------------------------------------------------
template <int M, int ADJ, int GRAD>
struct UL {
    using B = BX<M>;
    static constexpr bool IMG = ADJ == 2;
    static constexpr int NI = IMG ? 7 : 9 + (GRAD ? 3 : 0);
    static constexpr int OEY = 0, OFY = B::YS, OEZ = 2 * B::YS, OFZ = OEZ + B::ZS, OI = OFZ + B::ZS,
                         SZ = OI + NI * IS;
    // interior slots (ADJ = 2: lam_p, lam_r in PC, RC; g_eps, g_delta in UP, UR)
    static constexpr int QE = 0, QF = 1, MM = 2, PC = IMG ? 2 : 3, RC = PC + 1, PP = 5, RP = 6, EP = 7,
                         DE = IMG ? 4 : 8, UP = IMG ? 5 : 9, UR = UP + 1, GG = UP + 2;
    static constexpr uint32_t BYTES = 4u * (2 * B::YR * B::YC + 2 * B::ZR * B::ZC + NI * IS);
};

struct UMaps {
    CUtensorMap ey, fy, ez, fz, qe, qf, m, pc, rc, pp, rp, e, d, up, ur, g;
};

template <int M, int ADJ, int GRAD>
WP_DEV void tti_upd_body(const GridDev &g, const FDW &w, const float *__restrict__ ex,
                         const float *__restrict__ fx, const UMaps &mp, float *__restrict__ pp,
                         float *__restrict__ rp, float *__restrict__ grad, float *__restrict__ zp,
                         float *__restrict__ zr, int *flag, int check, int bx, int by, int bz, int xc, int *err)
{
    using L = UL<M, ADJ, GRAD>;
    using B = BX<M>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, warp = (ty * TZ2 + tz) >> 5, lane = (ty * TZ2 + tz) & 31;
    const bool lead = warp == 0 && lane == 0;
    const int z0 = bx * FZ, y0 = by * FY;
    const int z = z0 + 2 * tz, y = y0 + ty;
    const int xa = bz * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        float *I = S + L::OI;
        uint64_t *bar = &bars[st];
        mbar_expect(bar, L::BYTES);
        tma3(S + L::OEY, &mp.ey, z0, y0 - M, x, bar);
        tma3(S + L::OFY, &mp.fy, z0, y0 - M, x, bar);
        tma3(S + L::OEZ, &mp.ez, z0 - B::MZ, y0, x, bar);
        tma3(S + L::OFZ, &mp.fz, z0 - B::MZ, y0, x, bar);
        tma3(I + L::QE * IS, &mp.qe, z0, y0, x + M, bar);             // beyond NX: zeros
        tma3(I + L::QF * IS, &mp.qf, z0, y0, x + M, bar);
        tma3(I + L::PC * IS, &mp.pc, z0, y0, x, bar);
        tma3(I + L::RC * IS, &mp.rc, z0, y0, x, bar);
        tma3(I + L::DE * IS, &mp.d, z0, y0, x, bar);
        if (L::IMG) {
            tma3(I + L::UP * IS, &mp.up, z0, y0, x, bar);
            tma3(I + L::UR * IS, &mp.ur, z0, y0, x, bar);
        } else {
            tma3(I + L::MM * IS, &mp.m, z0, y0, x, bar);
            tma3(I + L::PP * IS, &mp.pp, z0, y0, x, bar);
            tma3(I + L::RP * IS, &mp.rp, z0, y0, x, bar);
            tma3(I + L::EP * IS, &mp.e, z0, y0, x, bar);
            if (GRAD) {
                tma3(I + L::UP * IS, &mp.up, z0, y0, x, bar);
                tma3(I + L::UR * IS, &mp.ur, z0, y0, x, bar);
                tma3(I + L::GG * IS, &mp.g, z0, y0, x, bar);
            }
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
    float2 qe[Q], qf[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        const int xq = xa - M + j;
        const bool in = act && xq >= 0 && xq < g.NX;
        qe[j] = in ? ldg2(ex, xq * pl + q0) : Z2;
        qf[j] = in ? ldg2(fx, xq * pl + q0) : Z2;
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
        qe[Q - 1] = lds2(I + L::QE * IS);
        qf[Q - 1] = lds2(I + L::QF * IS);
        if (act) {
            const float *sey = S + L::OEY, *sfy = S + L::OFY;
            float we[2 * M + 2], wf[2 * M + 2];
            zwin<M>(S + L::OEZ + izr, cz, we);
            zwin<M>(S + L::OFZ + izr, cz, wf);
            float h0a = 0.f, h0b = 0.f, hza = 0.f, hzb = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                const float2 ex_ = dif2(qe[M + k], qe[M - k]), fx_ = dif2(qf[M + k], qf[M - k]);
                const float2 ey_ = dif2(lds2(sey + iy + k * B::YC), lds2(sey + iy - k * B::YC));
                const float2 fy_ = dif2(lds2(sfy + iy + k * B::YC), lds2(sfy + iy - k * B::YC));
                h0a += c * (ex_.x + ey_.x + (we[M + k] - we[M - k]));
                h0b += c * (ex_.y + ey_.y + (we[M + k + 1] - we[M - k + 1]));
                hza += c * (fx_.x + fy_.x + (wf[M + k] - wf[M - k]));
                hzb += c * (fx_.y + fy_.y + (wf[M + k + 1] - wf[M - k + 1]));
            }
            const unsigned q = x * pl + q0;
            if (L::IMG) {
                const float2 lp = lds2(I + L::PC * IS), lr = lds2(I + L::RC * IS), d_ = lds2(I + L::DE * IS);
                const float2 ge = lds2(I + L::UP * IS), gd = lds2(I + L::UR * IS);
                const float h0a_ = h0a * g.ih, h0b_ = h0b * g.ih, hza_ = hza * g.ih, hzb_ = hzb * g.ih;
                st2(grad, q, ge.x + 2.f * dt2 * lp.x * h0a_, ge.y + 2.f * dt2 * lp.y * h0b_);
                st2(zp, q, gd.x + dt2 * (lp.x * hza_ + lr.x * h0a_) / sqrtf(1.f + 2.f * d_.x),
                    gd.y + dt2 * (lp.y * hzb_ + lr.y * h0b_) / sqrtf(1.f + 2.f * d_.y));
            } else {
                const float2 mm = lds2(I + L::MM * IS), p1 = lds2(I + L::PC * IS), r1 = lds2(I + L::RC * IS);
                const float2 p0 = lds2(I + L::PP * IS), r0 = lds2(I + L::RP * IS);
                const float2 e_ = lds2(I + L::EP * IS), d_ = lds2(I + L::DE * IS);
                const float sxv = __ldg(sx + x);
                const float h0[2] = {h0a * g.ih, h0b * g.ih}, hz[2] = {hza * g.ih, hzb * g.ih};
                const float M2[2] = {mm.x, mm.y}, E2[2] = {e_.x, e_.y}, D2[2] = {d_.x, d_.y};
                const float P1[2] = {p1.x, p1.y}, R1[2] = {r1.x, r1.y}, P0[2] = {p0.x, p0.y}, R0[2] = {r0.x, r0.y};
                const float SYZ[2] = {syz0, syz1};
                float pn[2], rn[2], Lp[2], Lr[2], c1[2], c2[2];
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    c1[i] = 1.f + 2.f * E2[i];
                    c2[i] = sqrtf(1.f + 2.f * D2[i]);
                    if (!ADJ) {
                        Lp[i] = c1[i] * h0[i] + c2[i] * hz[i];
                        Lr[i] = c2[i] * h0[i] + hz[i];
                    } else {
                        Lp[i] = h0[i];
                        Lr[i] = hz[i];
                    }
                    const float sd = hdt * (sxv + SYZ[i]);
                    const float A = M2[i] * (1.f + sd), Bc = M2[i] * (1.f - sd);
                    pn[i] = (dt2 * Lp[i] + 2.f * M2[i] * P1[i] - Bc * P0[i]) / A;
                    rn[i] = (dt2 * Lr[i] + 2.f * M2[i] * R1[i] - Bc * R0[i]) / A;
                }
                st2(pp, q, pn[0], pn[1]);
                st2(rp, q, rn[0], rn[1]);
                if (ADJ) {
                    st2(zp, q, c1[0] * pn[0] + c2[0] * rn[0], c1[1] * pn[1] + c2[1] * rn[1]);
                    st2(zr, q, c2[0] * pn[0] + rn[0], c2[1] * pn[1] + rn[1]);
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
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qe[j] = qe[j + 1];
            qf[j] = qf[j + 1];
        }
        R.release(lane);
    }
}

template <int M, int ADJ, int GRAD>
__global__ void __launch_bounds__(NTP, occ(2))
tti_upd_tma(GridDev g, FDW w, const float *__restrict__ ex, const float *__restrict__ fx,
            const __grid_constant__ UMaps mp, float *__restrict__ pp, float *__restrict__ rp,
            float *__restrict__ grad, float *__restrict__ zp, float *__restrict__ zr, int *flag, int check,
            int xc, int *err)
{
    tti_upd_body<M, ADJ, GRAD>(g, w, ex, fx, mp, pp, rp, grad, zp, zr, flag, check, blockIdx.x, blockIdx.y,
                               blockIdx.z, xc, err);
}

// ---------------------------------------------------------------------------
// Batched shots (Sec. III-B: many independent experiments): one launch of
// each pass serves every shot of a wave.  Each CTA takes its tile
// (shot, z tile, y tile, x chunk) from a table and its shot's grid, arrays
// and tensor maps from a per-shot entry in device memory (the maps are
// encoded on the host before the launch and never change during it).
// ---------------------------------------------------------------------------
struct TtiShot {
    RMaps rm;
    UMaps um;
    GridDev g;
    const float *rp, *rr;    // rotation input: (p, r), or zeta = C lam
    float *t[8];             // intermediates ex ey ez fx fy fz, zeta p, r
    float *pn, *rn;          // new level (written over the oldest)
    float *grad;
    int *flag;
    int check, xc;
};

template <int M>
__global__ void __launch_bounds__(NTP, occ(2))
tti_rot_batch(const TtiShot *__restrict__ shots, const int4 *__restrict__ tiles, FDW w)
{
    const int4 tl = tiles[blockIdx.x];
    const TtiShot &S = shots[tl.x];
    tti_rot_body<M, 0>(S.g, w, S.rp, S.rr, S.rm, S.t[0], S.t[1], S.t[2], S.t[3], S.t[4], S.t[5], F3{}, tl.y, tl.z,
                           tl.w, S.xc, S.flag);
}

template <int M, int ADJ, int GRAD>
__global__ void __launch_bounds__(NTP, occ(2))
tti_upd_batch(const TtiShot *__restrict__ shots, const int4 *__restrict__ tiles, FDW w)
{
    const int4 tl = tiles[blockIdx.x];
    const TtiShot &S = shots[tl.x];
    tti_upd_body<M, ADJ, GRAD>(S.g, w, S.t[0], S.t[3], S.um, S.pn, S.rn, S.grad, S.t[6], S.t[7], S.flag, S.check,
                               tl.y, tl.z, tl.w, S.xc, S.flag);
}

// ---------------------------------------------------------------------------
// Isotropic acoustic step (Sec. II-A, Eq. acou; u.laplace of the
// wave-equation listing), with w = dt^2 / m:
//   u^{n+1} = (w L u^n + 2 u^n - (1 - sd) u^{n-1}) / (1 + sd),  sd = sig dt / 2,
// L the sum over axes of the centred second derivative (the damped leapfrog
// A u^{n+1} = dt^2 L u^n + 2 m u^n - B u^{n-1} divided by m).  L is
// symmetric, so the transposed step is the same pass; GRAD fuses the imaging
// g -= w u_f (L lam) with the forward field u_f.  u^{n+1} overwrites u^{n-1}
// (each point is read before it is written, and only by its own thread).
// Tile 32 (z) x 32 (y): each consumer thread updates 2 z points on 2
// consecutive rows, so its z windows and y taps serve both rows, with
// paired FP32 arithmetic (__ffma2_rn and friends: per component the results
// of the scalar operations).  The x loop is unrolled over the queue length,
// so the x-derivative queues rotate by renaming instead of register moves.
// stage: [u^n rect (y, z halo)] [queue head u^n (x+M)] [w, u^{n-1} (plane x)]
//        (+ [u_f, g])
// ---------------------------------------------------------------------------
constexpr int AFY = 2 * FY;       // rows per CTA
constexpr int AIS = FZ * AFY;     // interior box (floats)

template <int M, int GRAD>
struct AL {
    static constexpr int MZ = (M + 3) & ~3;
    static constexpr int RR = AFY + 2 * M, RC = FZ + 2 * MZ, RS = al32(RR * RC);
    static constexpr int NI = 3 + (GRAD ? 2 : 0);
    static constexpr int OU = 0, OI = RS, SZ = OI + NI * AIS;
    static constexpr int QH = 0, WW = 1, U0 = 2, UF = 3, GG = 4;
    static constexpr uint32_t BYTES = 4u * (RR * RC + NI * AIS);
    static constexpr int NS = GRAD ? 3 : 4;   // ring stages that still fit two CTAs per SM
};

struct AMaps {
    CUtensorMap u, q, w, u0, uf, g;
};

template <int M, int GRAD>
__global__ void __launch_bounds__(NTP, M <= 6 ? 2 : 1)
acu_tma(GridDev g, FDW w, const float *__restrict__ u1, float *__restrict__ u0, float *__restrict__ grad,
        const __grid_constant__ AMaps mp, int *flag, int check, int xc, int *err)
{
    using L = AL<M, GRAD>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::NS * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, lane = (ty * TZ2 + tz) & 31;
    const bool lead = ty == 0 && tz == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * AFY;
    const int z = z0 + 2 * tz, ya = y0 + 2 * ty;          // rows ya, ya + 1
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX), nit = xb - xa;
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        float *I = S + L::OI;
        uint64_t *bar = &bars[st];
        mbar_expect(bar, L::BYTES);
        tma3(S + L::OU, &mp.u, z0 - L::MZ, y0 - M, x, bar);
        tma3(I + L::QH * AIS, &mp.q, z0, y0, x + M, bar);             // beyond NX: zeros
        tma3(I + L::WW * AIS, &mp.w, z0, y0, x, bar);
        tma3(I + L::U0 * AIS, &mp.u0, z0, y0, x, bar);
        if (GRAD) {
            tma3(I + L::UF * AIS, &mp.uf, z0, y0, x, bar);
            tma3(I + L::GG * AIS, &mp.g, z0, y0, x, bar);
        }
    };
    RingN<L::NS> R(bars);
    if (lead) {
        R.init();
        ck_begin(g.N, err);
    }
    __syncthreads();
    if (ty >= FY) {                                       // producer warp
        if (lane == 0) R.produce(xa, nit, issue, err);
        return;
    }
    const bool a0 = ya < g.NY && z < g.NZ, a1 = a0 && ya + 1 < g.NY;
    const unsigned pl = (unsigned)g.NY * (unsigned)g.NZ;
    const unsigned qa = a0 ? (unsigned)ya * g.NZ + z : 0u, qb = a1 ? qa + g.NZ : 0u;
    const float2 Z2 = make_float2(0.f, 0.f);
    float2 qu0[Q], qu1[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        const int xq = xa - M + j;
        const bool in = xq >= 0 && xq < g.NX;
        qu0[j] = a0 && in ? ldg2(u1, xq * pl + qa) : Z2;
        qu1[j] = a1 && in ? ldg2(u1, xq * pl + qb) : Z2;
    }
    const float *sx = g.tab, *sy = g.tab + g.NX, *sz = g.tab + g.NX + g.NY;
    const float sz0 = a0 ? __ldg(sz + z) : 0.f, sz1 = a0 ? __ldg(sz + z + 1) : 0.f;
    const float sy0 = a0 ? __ldg(sy + ya) : 0.f, sy1 = a1 ? __ldg(sy + ya + 1) : 0.f;
    const float2 syz[2] = {make_float2(sy0 + sz0, sy0 + sz1), make_float2(sy1 + sz0, sy1 + sz1)};
    const float hdt = 0.5f * g.dt;
    const float2 c0v = f2s(3.f * w.d2[0]), ih2 = f2s(g.ih * g.ih), one = f2s(1.f), two = f2s(2.f),
                 mone = f2s(-1.f);
    const int cz = L::MZ + 2 * tz, ii = 2 * ty * FZ + 2 * tz, cr = 2 * ty;
    const unsigned qr[2] = {qa, qb};
    const bool ar[2] = {a0, a1};
    for (int x0 = xa; x0 < xb; x0 += Q) {
#pragma unroll
        for (int s = 0; s < Q; s++) {
            const int x = x0 + s;
            if (x >= xb) break;
            if (!__all_sync(0xffffffffu, R.wait_full())) {
                if (lane == 0) atomicOr(err, 2);
                return;
            }
            const float *S = sm + R.st * L::SZ;
            const float *I = S + L::OI + ii;
            qu0[(s + 2 * M) % Q] = lds2(I + L::QH * AIS);
            qu1[(s + 2 * M) % Q] = lds2(I + L::QH * AIS + FZ);
            if (a0) {
                const float *su = S + L::OU;
                float2 col[2 * M + 2];               // y taps of both rows: rect rows cr .. cr+2M+1
#pragma unroll
                for (int i = 0; i < 2 * M + 2; i++) col[i] = lds2(su + (cr + i) * L::RC + cz);
                float2 lap[2];
#pragma unroll
                for (int r = 0; r < 2; r++) {
                    const float2 *qu = r ? qu1 : qu0;
                    float wz[2 * M + 2];
                    zwin<M>(su + (cr + M + r) * L::RC, cz, wz);
                    float2 acc = f2mul(c0v, col[M + r]);
#pragma unroll
                    for (int k = 1; k <= M; k++) {
                        const float2 sxk = f2add(qu[(s + M + k) % Q], qu[(s + M - k) % Q]);
                        const float2 syk = f2add(col[M + r + k], col[M + r - k]);
                        const float2 szk = make_float2(wz[M + k] + wz[M - k], wz[M + k + 1] + wz[M - k + 1]);
                        acc = f2fma(f2s(w.d2[k]), f2add(f2add(sxk, syk), szk), acc);
                    }
                    lap[r] = f2mul(acc, ih2);
                }
                const float2 sxv = f2s(__ldg(sx + x));
#pragma unroll
                for (int r = 0; r < 2; r++) {
                    if (!ar[r]) continue;
                    const float2 wv = lds2(I + L::WW * AIS + r * FZ), p0 = lds2(I + L::U0 * AIS + r * FZ);
                    const float2 sd = f2mul(f2s(hdt), f2add(sxv, syz[r]));
                    float2 num = f2mul(wv, lap[r]);
                    num = f2fma(two, col[M + r], num);
                    num = f2fma(f2add(sd, mone), p0, num);
                    const float2 den = f2add(one, sd);
                    const float2 un = make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
                    const unsigned q = x * pl + qr[r];
                    st2(u0, q, un.x, un.y);
                    if (GRAD) {
                        const float2 uf = lds2(I + L::UF * AIS + r * FZ), gg = lds2(I + L::GG * AIS + r * FZ);
                        const float2 t = f2fma(f2mul(mone, wv), uf, Z2);
                        const float2 gn = f2fma(t, lap[r], gg);
                        st2(grad, q, gn.x, gn.y);
                    }
                    if (check && !(isfinite(un.x) && isfinite(un.y))) atomicOr(flag, 1);
                }
            }
            R.release(lane);
        }
    }
}


// descriptors of the velocity pass: velocities v[3], stress-like fields
// sig[6] (xx yy zz xy xz yz)
template <int M>
bool vmaps(prop_s *P, float *const *v, float *const *sig, VMaps *m)
{
    using B = BX<M>;
    bool ok = map_of(P, sig[3], B::YC, B::YR, &m->xy) && map_of(P, sig[1], B::YC, B::YR, &m->yy) &&
              map_of(P, sig[4], B::ZC, B::ZR, &m->xz) && map_of(P, sig[2], B::ZC, B::ZR, &m->zz) &&
              map_of(P, sig[5], B::RC, B::RR, &m->yz) && map_of(P, P->bu, B::PC, B::PR, &m->b) &&
              map_of(P, sig[0], FZ, FY, &m->qxx) && map_of(P, sig[3], FZ, FY, &m->qxy) &&
              map_of(P, sig[4], FZ, FY, &m->qxz) && map_of(P, P->bu, FZ, FY, &m->bi);
    for (int i = 0; i < 3; i++) ok = ok && map_of(P, v[i], FZ, FY, &m->v[i]);
    return ok;
}
// descriptors of the stress pass: velocities vel[3], stress-like interiors t[6]
template <int M>
bool tmaps(prop_s *P, const float *const *vel, const float *const *t, TMaps *m)
{
    using B = BX<M>;
    bool ok = map_of(P, vel[0], B::RC, B::RR, &m->vx) && map_of(P, vel[1], B::RC, B::RR, &m->vy) &&
              map_of(P, vel[2], B::RC, B::RR, &m->vz) && map_of(P, P->mu, B::PC, B::PR, &m->mu) &&
              map_of(P, P->lam, FZ, FY, &m->lam) && map_of(P, vel[0], FZ, FY, &m->qvx) &&
              map_of(P, vel[1], FZ, FY, &m->qvy) && map_of(P, vel[2], FZ, FY, &m->qvz);
    for (int i = 0; i < 6; i++) ok = ok && map_of(P, t[i], FZ, FY, &m->t[i]);
    return ok;
}

dim3 el_grid(const prop_s *P)
{
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    return dim3((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
}

template <int M, int ADJ>
int launch_v(prop_s *P, const GridDev &g, const F9 &s, const F5 &o, const VMaps &vm)
{
    const size_t sm = NSTAGE * VL<M>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(el_vpass_tma<M, ADJ>, sm);
    (void)attr;
    el_vpass_tma<M, ADJ><<<el_grid(P), dim3(TZ2, FY + 2, 1), sm, P->stream>>>(g, P->w, s, o, vm, P->xchunk,
                                                                                P->flag);
    P->kern_launches++;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}
template <int M, int MODE>
int launch_t(prop_s *P, const GridDev &g, const F9 &s, const F5 &o, const TMaps &tm)
{
    const size_t sm = NSTAGE * TL<M, MODE>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(el_tpass_tma<M, MODE>, sm);
    (void)attr;
    el_tpass_tma<M, MODE><<<el_grid(P), dim3(TZ2, FY + 2, 1), sm, P->stream>>>(g, P->w, s, o, tm, P->xchunk,
                                                                                 P->flag);
    P->kern_launches++;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

template <int M>
int el_launch(prop_s *P, float *const *S, float dt)
{
    GridDev g = P->g;
    g.dt = dt;
    F9 s;
    for (int i = 0; i < 9; i++) s.f[i] = S[i];
    const F5 o{};
    VMaps vm;
    TMaps tm;
    if (!vmaps<M>(P, S, S + 3, &vm) || !tmaps<M>(P, S, S + 3, &tm))
        return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    WP_TRY((launch_v<M, 0>(P, g, s, o, vm)));
    return launch_t<M, 0>(P, g, s, o, tm);
}

// transposed step in the tbar form with imaging (one forward step k -> k+1):
// on entry S[3..8] = t = g tbar and sig[0..5] = C t; S[0..2] = vbar.
//   vbar <- g (vbar - dt Dtau(sig)),  w = b_avg vbar   (w[0..2])
//   g_lambda, g_mu, edge products from t and S(v^{k+1})
//   tbar <- t - dt S(w)
template <int M>
int el_adj_grad(prop_s *P, float *const *S, float *const *sig, float *const *w, const float *const *v1,
                float *const *gr, float *const *ep)
{
    const GridDev &g = P->g;
    VMaps vm;
    TMaps tg, tt;
    if (!vmaps<M>(P, S, sig, &vm) || !tmaps<M>(P, v1, S + 3, &tg) || !tmaps<M>(P, w, S + 3, &tt) ||
        !map_of(P, gr[0], FZ, FY, &tg.gl) || !map_of(P, gr[1], FZ, FY, &tg.gm))
        return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    F9 sv, sg, st;
    for (int i = 0; i < 3; i++) {
        sv.f[i] = S[i];
        sg.f[i] = const_cast<float *>(v1[i]);
        st.f[i] = w[i];
    }
    for (int i = 0; i < 6; i++) {
        sv.f[3 + i] = sig[i];
        sg.f[3 + i] = S[3 + i];
        st.f[3 + i] = S[3 + i];
    }
    const F5 ow{{w[0], w[1], w[2], nullptr, nullptr}}, og{{gr[0], gr[1], ep[0], ep[1], ep[2]}}, none{};
    WP_TRY((launch_v<M, 1>(P, g, sv, ow, vm)));
    WP_TRY((launch_t<M, 2>(P, g, sg, og, tg)));
    return launch_t<M, 1>(P, g, st, none, tt);
}

template <int M, int ADJ, int GRAD>
int tti_launch(prop_s *P, float *const *S, const float *up, const float *ur, float *grad)
{
    using B = BX<M>;
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ2, FY + 2, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    // the rotation pass differentiates (p, r), or zeta = C lam (tmp[6], tmp[7])
    // in the transposed step
    const float *rp_ = ADJ ? t[6] : S[0], *rr_ = ADJ ? t[7] : S[1];
    RMaps rm;
    UMaps um;
    bool ok = map_of(P, rp_, B::RC, B::RR, &rm.p) && map_of(P, rr_, B::RC, B::RR, &rm.r) &&
              map_of(P, rp_, FZ, FY, &rm.qp) && map_of(P, rr_, FZ, FY, &rm.qr) &&
              map_of(P, P->nrm[0], FZ, FY, &rm.nx) && map_of(P, P->nrm[1], FZ, FY, &rm.ny) &&
              map_of(P, t[1], B::YC, B::YR, &um.ey) && map_of(P, t[4], B::YC, B::YR, &um.fy) &&
              map_of(P, t[2], B::ZC, B::ZR, &um.ez) && map_of(P, t[5], B::ZC, B::ZR, &um.fz) &&
              map_of(P, t[0], FZ, FY, &um.qe) && map_of(P, t[3], FZ, FY, &um.qf) &&
              map_of(P, P->m, FZ, FY, &um.m) && map_of(P, S[0], FZ, FY, &um.pc) &&
              map_of(P, S[1], FZ, FY, &um.rc) && map_of(P, S[2], FZ, FY, &um.pp) &&
              map_of(P, S[3], FZ, FY, &um.rp) && map_of(P, P->eps, FZ, FY, &um.e) &&
              map_of(P, P->del, FZ, FY, &um.d);
    if (GRAD)
        ok = ok && map_of(P, up, FZ, FY, &um.up) && map_of(P, ur, FZ, FY, &um.ur) &&
             map_of(P, grad, FZ, FY, &um.g);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = RL<M>::NS * RL<M>::SZ * sizeof(float) + 64,
                 s2 = NSTAGE * UL<M, ADJ, GRAD>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_rot_tma<M>, s1) && set_smem(tti_upd_tma<M, ADJ, GRAD>, s2);
    (void)attr;
    tti_rot_tma<M><<<grd, blk, s1, P->stream>>>(g, P->w, rp_, rr_, rm, t[0], t[1], t[2], t[3], t[4], t[5], F3{},
                                               xc, P->flag);
    tti_upd_tma<M, ADJ, GRAD><<<grd, blk, s2, P->stream>>>(g, P->w, t[0], t[3], um, S[2], S[3], grad, t[6], t[7],
                                                          P->flag, P->d.check_nan, xc, P->flag);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

// Tilt/azimuth imaging of one step.  With zeta = C lam (dz: D zeta_p, D zeta_r)
// and the forward field's g = D p, h = D r (du), the step's term of dJ/dn is
//   V = D zeta_p (n.g) + (n.D zeta_p) g - D zeta_r (n.h) - (n.D zeta_r) h
// (the derivative of -zeta_p^T (I - n n^T) g - (n.D zeta_r)(n.h), the
// bilinear forms of H0 and Hz, with respect to n at the point);
// acc += s V, s = dt^2.  n is the stored axis (n_z >= 0).
struct AxisIn {
    const float *dz[6], *du[6], *nx, *ny;
    float *acc[3];
};
__global__ void tti_axis_image(long long n, float s, AxisIn a)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
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
    for (int c = 0; c < 3; c++)
        a.acc[c][q] += s * (zp[c] * ng + nzp * gp[c] - zr[c] * nh - nzr * gr[c]);
}

// dJ/dn (stored axis) -> dJ/dtheta into a0, dJ/dphi into a1: with the sign sg
// that makes n_z >= 0, the stored axis is sg n(theta, phi), so
// dJ/dt = sg dn/dt . acc  (t = theta, phi)
__global__ void tti_axis_finalize(long long n, const float *th, const float *ph, float *a0, float *a1,
                                  const float *a2)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    double st, ct, sp, cp;
    sincos((double)th[q], &st, &ct);
    sincos((double)ph[q], &sp, &cp);
    const double sg = ct < 0.0 ? -1.0 : 1.0;
    const double v0 = a0[q], v1 = a1[q], v2 = a2[q];
    a0[q] = (float)(sg * (ct * cp * v0 + ct * sp * v1 - st * v2));
    a1[q] = (float)(sg * (-st * sp * v0 + st * cp * v1));
}

// imaging of the coupling matrix (eps, delta gradients) with the forward
// field (up, ur) at level n and the adjoint field (lp, lr) at level n+1:
// rotation pass on the forward field, then the update pass in mode 2.
// gax != NULL: also the tilt/azimuth term, from zeta = C lam in tmp[6], tmp[7]
// (raw rotation passes on zeta into tmp[0..5] and on the forward field into
// tmp[8..13], then tti_axis_image into gax[0..2])
template <int M>
int tti_image_aniso(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr, float *ge,
                    float *gd, float *const *gax)
{
    using B = BX<M>;
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ2, FY + 2, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    RMaps rm;
    UMaps um;
    bool ok = map_of(P, up, B::RC, B::RR, &rm.p) && map_of(P, ur, B::RC, B::RR, &rm.r) &&
              map_of(P, up, FZ, FY, &rm.qp) && map_of(P, ur, FZ, FY, &rm.qr) &&
              map_of(P, P->nrm[0], FZ, FY, &rm.nx) && map_of(P, P->nrm[1], FZ, FY, &rm.ny) &&
              map_of(P, t[1], B::YC, B::YR, &um.ey) && map_of(P, t[4], B::YC, B::YR, &um.fy) &&
              map_of(P, t[2], B::ZC, B::ZR, &um.ez) && map_of(P, t[5], B::ZC, B::ZR, &um.fz) &&
              map_of(P, t[0], FZ, FY, &um.qe) && map_of(P, t[3], FZ, FY, &um.qf) &&
              map_of(P, lp, FZ, FY, &um.pc) && map_of(P, lr, FZ, FY, &um.rc) &&
              map_of(P, P->del, FZ, FY, &um.d) && map_of(P, ge, FZ, FY, &um.up) && map_of(P, gd, FZ, FY, &um.ur);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = RL<M>::NS * RL<M>::SZ * sizeof(float) + 64, s2 = NSTAGE * UL<M, 2, 0>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_rot_tma<M>, s1) && set_smem(tti_upd_tma<M, 2, 0>, s2);
    (void)attr;
    tti_rot_tma<M><<<grd, blk, s1, P->stream>>>(g, P->w, up, ur, rm, t[0], t[1], t[2], t[3], t[4], t[5], F3{},
                                               xc, P->flag);
    tti_upd_tma<M, 2, 0><<<grd, blk, s2, P->stream>>>(g, P->w, t[0], t[3], um, nullptr, nullptr, ge, gd, nullptr,
                                                     P->flag, 0, xc, P->flag);
    P->kern_launches += 2;
    if (gax) {
        RMaps rz;
        ok = map_of(P, t[6], B::RC, B::RR, &rz.p) && map_of(P, t[7], B::RC, B::RR, &rz.r) &&
             map_of(P, t[6], FZ, FY, &rz.qp) && map_of(P, t[7], FZ, FY, &rz.qr) && (rz.nx = rm.nx, true) &&
             (rz.ny = rm.ny, true);
        if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
        static const bool attr_raw = set_smem(tti_rot_tma<M, 1>, s1);
        (void)attr_raw;
        tti_rot_tma<M, 1><<<grd, blk, s1, P->stream>>>(g, P->w, t[6], t[7], rz, t[0], t[1], t[2], t[3], t[4], t[5],
                                                       F3{}, xc, P->flag);
        tti_rot_tma<M, 1><<<grd, blk, s1, P->stream>>>(g, P->w, up, ur, rm, t[8], t[9], t[10], t[11], t[12], t[13],
                                                       F3{}, xc, P->flag);
        AxisIn ai;
        for (int c = 0; c < 6; c++) {
            ai.dz[c] = t[c];
            ai.du[c] = t[8 + c];
        }
        ai.nx = P->nrm[0];
        ai.ny = P->nrm[1];
        for (int c = 0; c < 3; c++) ai.acc[c] = gax[c];
        const long long n = (long long)g.N;
        tti_axis_image<<<(unsigned)((n + 255) / 256), 256, 0, P->stream>>>(n, P->g.dt * P->g.dt, ai);
        P->kern_launches += 3;
    }
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

template <int M>
int tti_launch_any(prop_s *P, float *const *S, bool adjoint, const float *up, const float *ur, float *grad)
{
    if (!adjoint) return tti_launch<M, 0, 0>(P, S, up, ur, grad);
    return grad ? tti_launch<M, 1, 1>(P, S, up, ur, grad) : tti_launch<M, 1, 0>(P, S, up, ur, grad);
}

// acoustic step: S[0] = u^n, S[1] = u^{n-1} (overwritten by u^{n+1});
// grad != NULL: imaging with the forward field uf
template <int M, int GRAD>
int acu_launch(prop_s *P, float *const *S, const float *uf, float *grad)
{
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ2, FY + 2, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + AFY - 1) / AFY, (g.NX + xc - 1) / xc);
    using L = AL<M, GRAD>;
    AMaps am;
    bool ok = map_of(P, S[0], L::RC, L::RR, &am.u) && map_of(P, S[0], FZ, AFY, &am.q) &&
              map_of(P, P->acw, FZ, AFY, &am.w) && map_of(P, S[1], FZ, AFY, &am.u0);
    if (GRAD) ok = ok && map_of(P, uf, FZ, AFY, &am.uf) && map_of(P, grad, FZ, AFY, &am.g);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t sb = AL<M, GRAD>::NS * AL<M, GRAD>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(acu_tma<M, GRAD>, sb);
    (void)attr;
    acu_tma<M, GRAD><<<grd, blk, sb, P->stream>>>(g, P->w, S[0], S[1], grad, am, P->flag, P->d.check_nan, xc,
                                                  P->flag);
    P->kern_launches += 1;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing
// completes, with a limit of limit_ns on %globaltimer, then reports bit 2
// (as a TMA pass whose copies never land) and returns.
__global__ void wait_probe(uint64_t limit_ns, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_init();
    }
    __syncwarp();
    bool ok = false;
    if (threadIdx.x == 0) {
        const uint64_t t0 = gtimer();
        while (!(ok = mbar_try(&bar, 0)) && gtimer() - t0 < limit_ns) {
        }
        if (!ok) atomicOr(err, 2);
    }
    __syncwarp();
}

// centred first derivatives of (p, r) and the half-point products of their
// staggered derivatives through the rotation pass in mode 2: dp[0..2] = D p,
// dr[0..2] = D r, h[0..2] = (D+ p)(D+ r) per axis
template <int M>
int raw_half(prop_s *P, const float *p, const float *r, float *const *dp, float *const *dr, float *const *h)
{
    using B = BX<M>;
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(TZ2, FY + 2, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    RMaps rm;
    const bool ok = map_of(P, p, B::RC, B::RR, &rm.p) && map_of(P, r, B::RC, B::RR, &rm.r) &&
                    map_of(P, p, FZ, FY, &rm.qp) && map_of(P, r, FZ, FY, &rm.qr) &&
                    map_of(P, P->nrm[0], FZ, FY, &rm.nx) && map_of(P, P->nrm[1], FZ, FY, &rm.ny);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = RL<M>::NS * RL<M>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_rot_tma<M, 2>, s1);
    (void)attr;
    tti_rot_tma<M, 2><<<grd, blk, s1, P->stream>>>(g, P->w, p, r, rm, dp[0], dp[1], dp[2], dr[0], dr[1], dr[2],
                                                   F3{{h[0], h[1], h[2]}}, xc, P->flag);
    P->kern_launches += 1;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// Entry points of one tile height carry its suffix (_y8, _y16, _y32); the
// unit of the default height also holds the dispatchers by the handle's
// tile_y and everything that exists once (batched launches, self-test,
// acoustic pass, raw derivatives of the staggered-pair imaging).
#if WP_TILE_Y == 8
#define WP_TILE_FN(name) name##_y8
#elif WP_TILE_Y == 32
#define WP_TILE_FN(name) name##_y32
#else
#define WP_TILE_FN(name) name##_y16
#endif

#if WP_TILE_Y == 16
// launch the wait self-test on the handle's stream (limit in seconds, <= 2)
int wait_probe_launch(prop_s *P, double seconds)
{
    const double s = seconds < 0.0 ? 0.0 : (seconds > 2.0 ? 2.0 : seconds);
    wait_probe<<<1, 32, 0, P->stream>>>((uint64_t)(s * 1e9), P->flag);
    P->kern_launches += 1;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

// acoustic step through the TMA-fed pass (see acu_launch)
int acu_launch_tma(prop_s *P, float *const *S, const float *uf, float *grad)
{
    const int id = grad ? 7 : 6;
    prof_begin(P, id);
    int rc;
    switch (P->M) {
    case 2: rc = grad ? acu_launch<2, 1>(P, S, uf, grad) : acu_launch<2, 0>(P, S, uf, grad); break;
    case 4: rc = grad ? acu_launch<4, 1>(P, S, uf, grad) : acu_launch<4, 0>(P, S, uf, grad); break;
    case 6: rc = grad ? acu_launch<6, 1>(P, S, uf, grad) : acu_launch<6, 0>(P, S, uf, grad); break;
    case 8: rc = grad ? acu_launch<8, 1>(P, S, uf, grad) : acu_launch<8, 0>(P, S, uf, grad); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, id);
    return rc;
}

// TMA-fed passes need 16-byte row strides (NZ a multiple of 4), the
// driver's tensor-map encoder and (TTI) the symmetry-axis arrays
bool tma_usable(const prop_s *P)
{
    return P->g.NZ % 4 == 0 && encode_fn() != nullptr && getenv("WAVEPROP_NO_TMA") == nullptr &&
           (P->d.kind != PROP_TTI || (P->nrm[0] && P->nrm[1]));
}

#endif  // WP_TILE_Y == 16

// elastic step with time step dt_sign * dt (forward: +1; adjoint modelling
// in (b_avg vbar, g C tbar) variables: -1)
int WP_TILE_FN(el_launch_tma)(prop_s *P, float *const *S, float dt_sign)
{
    prof_begin(P, dt_sign > 0 ? 2 : 5);
    int rc;
    switch (P->M) {
    case 2: rc = el_launch<2>(P, S, dt_sign * P->g.dt); break;
    case 4: rc = el_launch<4>(P, S, dt_sign * P->g.dt); break;
    case 6: rc = el_launch<6>(P, S, dt_sign * P->g.dt); break;
    case 8: rc = el_launch<8>(P, S, dt_sign * P->g.dt); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, dt_sign > 0 ? 2 : 5);
    return rc;
}

// eps, delta (and theta, phi) imaging of one transposed TTI step (see
// tti_image_aniso; centred operators)
int WP_TILE_FN(tti_image_aniso_tma)(prop_s *P, const float *up, const float *ur, const float *lp,
                                    const float *lr, float *ge, float *gd, float *const *gax)
{
    switch (P->M) {
    case 2: return tti_image_aniso<2>(P, up, ur, lp, lr, ge, gd, gax);
    case 4: return tti_image_aniso<4>(P, up, ur, lp, lr, ge, gd, gax);
    case 6: return tti_image_aniso<6>(P, up, ur, lp, lr, ge, gd, gax);
    case 8: return tti_image_aniso<8>(P, up, ur, lp, lr, ge, gd, gax);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

#if WP_TILE_Y == 16
// the pointwise tilt/azimuth term for any pass family (dz: raw derivatives of
// zeta = C lam, du: of the forward field; acc += dt^2 V)
void tti_axis_image_launch(prop_s *P, const float *const *dz, const float *const *du, float *const *acc)
{
    AxisIn ai;
    for (int c = 0; c < 6; c++) {
        ai.dz[c] = dz[c];
        ai.du[c] = du[c];
    }
    ai.nx = P->nrm[0];
    ai.ny = P->nrm[1];
    for (int c = 0; c < 3; c++) ai.acc[c] = acc[c];
    const long long n = (long long)P->g.N;
    tti_axis_image<<<(unsigned)((n + 255) / 256), 256, 0, P->stream>>>(n, P->g.dt * P->g.dt, ai);
    P->kern_launches += 1;
}

// dJ/dn accumulators (computational grid) -> dJ/dtheta in a[0], dJ/dphi in a[1]
void tti_axis_to_angles(prop_s *P, float *const *a)
{
    const long long n = (long long)P->g.N;
    tti_axis_finalize<<<(unsigned)((n + 255) / 256), 256, 0, P->stream>>>(n, P->th, P->ph, a[0], a[1], a[2]);
    P->kern_launches += 1;
}

#endif  // WP_TILE_Y == 16

// the TMA passes of one transposed elastic step with imaging (see el_adj_grad)
int WP_TILE_FN(el_adj_grad_tma)(prop_s *P, float *const *S, float *const *sig, float *const *w,
                                const float *const *v1, float *const *gr, float *const *ep)
{
    switch (P->M) {
    case 2: return el_adj_grad<2>(P, S, sig, w, v1, gr, ep);
    case 4: return el_adj_grad<4>(P, S, sig, w, v1, gr, ep);
    case 6: return el_adj_grad<6>(P, S, sig, w, v1, gr, ep);
    case 8: return el_adj_grad<8>(P, S, sig, w, v1, gr, ep);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

int WP_TILE_FN(tti_launch_tma)(prop_s *P, float *const *S, bool adjoint, const float *img_p,
                               const float *img_r, float *grad)
{
    prof_begin(P, adjoint ? 1 : 0);
    int rc;
    switch (P->M) {
    case 2: rc = tti_launch_any<2>(P, S, adjoint, img_p, img_r, grad); break;
    case 4: rc = tti_launch_any<4>(P, S, adjoint, img_p, img_r, grad); break;
    case 6: rc = tti_launch_any<6>(P, S, adjoint, img_p, img_r, grad); break;
    case 8: rc = tti_launch_any<8>(P, S, adjoint, img_p, img_r, grad); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, adjoint ? 1 : 0);
    return rc;
}

// largest dynamic shared memory of the passes a handle of this kind and
// order launches at this tile height
namespace {
template <int M>
size_t smem_need(int kind)
{
    auto b = [](int floats) { return (size_t)floats * sizeof(float) + 64; };
    if (kind == PROP_ELASTIC)
        return std::max({b(NSTAGE * VL<M>::SZ), b(NSTAGE * TL<M, 0>::SZ), b(NSTAGE * TL<M, 1>::SZ),
                         b(NSTAGE * TL<M, 2>::SZ)});
    return std::max({b(RL<M>::NS * RL<M>::SZ), b(NSTAGE * UL<M, 0, 0>::SZ), b(NSTAGE * UL<M, 1, 0>::SZ),
                     b(NSTAGE * UL<M, 1, 1>::SZ), b(NSTAGE * UL<M, 2, 0>::SZ)});
}
}  // namespace

// true if the passes of the handle's kind and order fit one CTA's shared
// memory at this tile height (elastic and centred TTI)
bool WP_TILE_FN(tile_fits)(const prop_s *P)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    size_t need = 0;
    switch (P->M) {
    case 2: need = smem_need<2>(P->d.kind); break;
    case 4: need = smem_need<4>(P->d.kind); break;
    case 6: need = smem_need<6>(P->d.kind); break;
    case 8: need = smem_need<8>(P->d.kind); break;
    default: return false;
    }
    return need <= (size_t)optin;
}

#if WP_TILE_Y == 16
// the other tile heights, compiled in their own units
#define WP_DECL_HEIGHT(sfx)                                                                                    \
    bool tile_fits##sfx(const prop_s *P);                                                                     \
    int el_launch_tma##sfx(prop_s *P, float *const *S, float dt_sign);                                        \
    int tti_image_aniso_tma##sfx(prop_s *P, const float *up, const float *ur, const float *lp,                \
                                 const float *lr, float *ge, float *gd, float *const *gax);                   \
    int el_adj_grad_tma##sfx(prop_s *P, float *const *S, float *const *sig, float *const *w,                  \
                             const float *const *v1, float *const *gr, float *const *ep);                     \
    int tti_launch_tma##sfx(prop_s *P, float *const *S, bool adjoint, const float *img_p,                     \
                            const float *img_r, float *grad);
WP_DECL_HEIGHT(_y8)
WP_DECL_HEIGHT(_y32)
#undef WP_DECL_HEIGHT

// dispatch on the handle's tile height (prop_s::tile_y, set by the autotuner)
bool tile_height_fits(const prop_s *P, int ty)
{
    if (P->d.kind != PROP_ELASTIC && !(P->d.kind == PROP_TTI && P->d.tti_operator == 0)) return ty == 16;
    // a 32-row CTA (17 warps) gets at most 96 registers per thread; the
    // elastic passes above space order 8 need 144-168 and would spill
    if (ty == 32 && P->d.kind == PROP_ELASTIC && P->M > 4) return false;
    switch (ty) {
    case 8: return tile_fits_y8(P);
    case 16: return tile_fits_y16(P);
    case 32: return tile_fits_y32(P);
    }
    return false;
}
int el_launch_tma(prop_s *P, float *const *S, float dt_sign)
{
    switch (P->tile_y) {
    case 8: return el_launch_tma_y8(P, S, dt_sign);
    case 32: return el_launch_tma_y32(P, S, dt_sign);
    }
    return el_launch_tma_y16(P, S, dt_sign);
}
int tti_image_aniso_tma(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr,
                        float *ge, float *gd, float *const *gax)
{
    if (P->d.tti_operator == 1) return tti_sp_image_aniso_tma(P, up, ur, lp, lr, ge, gd, gax);
    switch (P->tile_y) {
    case 8: return tti_image_aniso_tma_y8(P, up, ur, lp, lr, ge, gd, gax);
    case 32: return tti_image_aniso_tma_y32(P, up, ur, lp, lr, ge, gd, gax);
    }
    return tti_image_aniso_tma_y16(P, up, ur, lp, lr, ge, gd, gax);
}
int el_adj_grad_tma(prop_s *P, float *const *S, float *const *sig, float *const *w, const float *const *v1,
                    float *const *gr, float *const *ep)
{
    switch (P->tile_y) {
    case 8: return el_adj_grad_tma_y8(P, S, sig, w, v1, gr, ep);
    case 32: return el_adj_grad_tma_y32(P, S, sig, w, v1, gr, ep);
    }
    return el_adj_grad_tma_y16(P, S, sig, w, v1, gr, ep);
}
int tti_launch_tma(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                   float *grad)
{
    switch (P->tile_y) {
    case 8: return tti_launch_tma_y8(P, S, adjoint, img_p, img_r, grad);
    case 32: return tti_launch_tma_y32(P, S, adjoint, img_p, img_r, grad);
    }
    return tti_launch_tma_y16(P, S, adjoint, img_p, img_r, grad);
}

// ---------------------------------------------------------------------------
// batched TTI steps: tables and launches
// ---------------------------------------------------------------------------
struct TtiBatch {
    // tile table (shot, z tile, y tile, x chunk), rebuilt when the shots'
    // shapes or x-extents change; shots with more tiles first, so the
    // longest work starts first
    std::vector<long long> sig;
    std::vector<int4> htiles;
    int4 *dtiles = nullptr;
    size_t tiles_cap = 0;
    // per-shot entries: device buffer, and pinned host staging in a ring of
    // slots (a slot is refilled only after its copy has run)
    TtiShot *dshots = nullptr;
    size_t shots_cap = 0;
    static constexpr int NSLOT = 8;
    TtiShot *hshots[NSLOT] = {};
    cudaEvent_t copied[NSLOT] = {};
    size_t hcap = 0;
    unsigned long long calls = 0;
    // elastic entries (bytes: one table for a modelling step, three for a
    // transposed step with imaging)
    void *del = nullptr;
    size_t del_cap = 0;
    char *hel[NSLOT] = {};
    size_t hel_cap = 0;
    cudaEvent_t elcopied[NSLOT] = {};
    // fixed tables of step configurations, one per slot (graph replay); the
    // mode of a slot: 0 forward step, 1 transposed step, 2 transposed step
    // with imaging
    std::vector<TtiShot *> dfixed;
    std::vector<int> fixed_mode;
    size_t fixed_cap = 0;
    int fixed_n = 0, fixed_M = 0;
    // fixed tables of elastic steps (graph replay): per slot n entries (a
    // forward step) or 3n (a transposed step with imaging)
    std::vector<ElShot *> elfixed;
    std::vector<int> elfixed_mode;
    size_t elfixed_cap = 0;
    FDW w{};
};

TtiBatch *tti_batch_new() { return new TtiBatch(); }

void tti_batch_free(TtiBatch *b)
{
    if (!b) return;
    cudaFree(b->dtiles);
    cudaFree(b->dshots);
    for (auto d : b->dfixed) cudaFree(d);
    for (auto d : b->elfixed) cudaFree(d);
    cudaFree(b->del);
    for (int i = 0; i < TtiBatch::NSLOT; i++) {
        if (b->elcopied[i]) {
            cudaEventSynchronize(b->elcopied[i]);
            cudaEventDestroy(b->elcopied[i]);
        }
        cudaFreeHost(b->hel[i]);
    }
    for (int i = 0; i < TtiBatch::NSLOT; i++) {
        if (b->copied[i]) {
            cudaEventSynchronize(b->copied[i]);
            cudaEventDestroy(b->copied[i]);
        }
        cudaFreeHost(b->hshots[i]);
    }
    delete b;
}

bool tti_batchable(const prop_s *P)
{
    return P->d.kind == PROP_TTI && P->d.tti_operator == 0 && tma_usable(P);
}

// per-shot entries of one step of every request into H[0..n)
template <int M, int ADJ, int GRAD>
int tti_batch_fill(const TtiBatchReq *req, int n, TtiShot *H, std::string *err)
{
    using B = BX<M>;
    for (int i = 0; i < n; i++) {
        prop_s *P = req[i].P;
        float *const *S = req[i].S;
        float *const *t = P->tmp;
        TtiShot &e = H[i];
        const float *rp_ = ADJ ? t[6] : S[0], *rr_ = ADJ ? t[7] : S[1];
        bool ok = map_of(P, rp_, B::RC, B::RR, &e.rm.p) && map_of(P, rr_, B::RC, B::RR, &e.rm.r) &&
                  map_of(P, rp_, FZ, FY, &e.rm.qp) && map_of(P, rr_, FZ, FY, &e.rm.qr) &&
                  map_of(P, P->nrm[0], FZ, FY, &e.rm.nx) && map_of(P, P->nrm[1], FZ, FY, &e.rm.ny) &&
                  map_of(P, t[1], B::YC, B::YR, &e.um.ey) && map_of(P, t[4], B::YC, B::YR, &e.um.fy) &&
                  map_of(P, t[2], B::ZC, B::ZR, &e.um.ez) && map_of(P, t[5], B::ZC, B::ZR, &e.um.fz) &&
                  map_of(P, t[0], FZ, FY, &e.um.qe) && map_of(P, t[3], FZ, FY, &e.um.qf) &&
                  map_of(P, P->m, FZ, FY, &e.um.m) && map_of(P, S[0], FZ, FY, &e.um.pc) &&
                  map_of(P, S[1], FZ, FY, &e.um.rc) && map_of(P, S[2], FZ, FY, &e.um.pp) &&
                  map_of(P, S[3], FZ, FY, &e.um.rp) && map_of(P, P->eps, FZ, FY, &e.um.e) &&
                  map_of(P, P->del, FZ, FY, &e.um.d);
        if (GRAD)
            ok = ok && map_of(P, req[i].up, FZ, FY, &e.um.up) && map_of(P, req[i].ur, FZ, FY, &e.um.ur) &&
                 map_of(P, req[i].grad, FZ, FY, &e.um.g);
        if (!ok) {
            *err = "cuTensorMapEncodeTiled failed";
            return PROP_ECUDA;
        }
        e.g = P->g;
        e.rp = rp_;
        e.rr = rr_;
        for (int k = 0; k < 8; k++) e.t[k] = t[k];
        e.pn = S[2];
        e.rn = S[3];
        e.grad = req[i].grad;
        e.flag = P->flag;
        e.check = P->d.check_nan;
        e.xc = P->xchunk;
    }
    return PROP_OK;
}

template <int M, int ADJ, int GRAD>
int tti_batch_launch(TtiBatch *b, const TtiBatchReq *req, int n, cudaStream_t st, std::string *err)
{
    // per-shot entries into the next staging slot
    const int slot = (int)(b->calls++ % TtiBatch::NSLOT);
    if (b->copied[slot] && cudaEventSynchronize(b->copied[slot]) != cudaSuccess) {
        *err = "batched TTI step: staging wait failed";
        return PROP_ECUDA;
    }
    TtiShot *H = b->hshots[slot];
    if (int rc = tti_batch_fill<M, ADJ, GRAD>(req, n, H, err)) return rc;
    auto ck = [&](cudaError_t c, const char *what) {
        if (c == cudaSuccess) return PROP_OK;
        *err = std::string("CUDA error '") + cudaGetErrorString(c) + "' in " + what;
        return c == cudaErrorMemoryAllocation ? PROP_ENOMEM : PROP_ECUDA;
    };
    if (int rc = ck(cudaMemcpyAsync(b->dshots, H, n * sizeof(TtiShot), cudaMemcpyHostToDevice, st),
                    "batched TTI step: shot table copy"))
        return rc;
    if (int rc = ck(cudaEventRecord(b->copied[slot], st), "batched TTI step: event")) return rc;
    const size_t s1 = RL<M>::NS * RL<M>::SZ * sizeof(float) + 64,
                 s2 = NSTAGE * UL<M, ADJ, GRAD>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_rot_batch<M>, s1) && set_smem(tti_upd_batch<M, ADJ, GRAD>, s2);
    (void)attr;
    const unsigned nt = (unsigned)b->htiles.size();
    const dim3 blk(TZ2, FY + 2, 1);
    tti_rot_batch<M><<<nt, blk, s1, st>>>(b->dshots, b->dtiles, req[0].P->w);
    tti_upd_batch<M, ADJ, GRAD><<<nt, blk, s2, st>>>(b->dshots, b->dtiles, req[0].P->w);
    for (int i = 0; i < n; i++) req[i].P->kern_launches += 2;
    return ck(cudaGetLastError(), "batched TTI step launch");
}

// tile table over the shots (cached while their shapes and x-extents stay
// the same); shots with more points first
static int batch_tiles(TtiBatch *b, const std::vector<prop_s *> &Ps, cudaStream_t st, std::string *err);
static int tti_batch_tiles(TtiBatch *b, const TtiBatchReq *req, int n, cudaStream_t st, std::string *err)
{
    std::vector<prop_s *> Ps(n);
    for (int i = 0; i < n; i++) Ps[i] = req[i].P;
    return batch_tiles(b, Ps, st, err);
}
static int batch_tiles(TtiBatch *b, const std::vector<prop_s *> &Ps, cudaStream_t st, std::string *err)
{
    const int n = (int)Ps.size();
    auto ck = [&](cudaError_t c, const char *what) {
        if (c == cudaSuccess) return PROP_OK;
        *err = std::string("CUDA error '") + cudaGetErrorString(c) + "' in " + what;
        return c == cudaErrorMemoryAllocation ? PROP_ENOMEM : PROP_ECUDA;
    };
    std::vector<long long> sig;
    for (int i = 0; i < n; i++) {
        const GridDev &g = Ps[i]->g;
        sig.insert(sig.end(), {(long long)g.NX, (long long)g.NY, (long long)g.NZ, (long long)Ps[i]->xchunk});
    }
    if (sig == b->sig) return PROP_OK;
    std::vector<std::pair<long long, int>> order;
    for (int i = 0; i < n; i++) order.emplace_back(-Ps[i]->g.N, i);
    std::stable_sort(order.begin(), order.end());
    b->htiles.clear();
    for (auto &o : order) {
        const int i = o.second;
        const GridDev &g = Ps[i]->g;
        const int xc = Ps[i]->xchunk;
        const int tz = (g.NZ + FZ - 1) / FZ, tyy = (g.NY + FY - 1) / FY, tx = (g.NX + xc - 1) / xc;
        for (int c = 0; c < tx; c++)
            for (int y = 0; y < tyy; y++)
                for (int z = 0; z < tz; z++) b->htiles.push_back(make_int4(i, z, y, c));
    }
    if (b->htiles.size() > b->tiles_cap) {
        cudaFree(b->dtiles);
        b->dtiles = nullptr;
        b->tiles_cap = 0;
        if (int rc = wp_dev_alloc((void **)&b->dtiles, b->htiles.size() * sizeof(int4), "batched TTI tile table",
                                  err))
            return rc;
        b->tiles_cap = b->htiles.size();
    }
    if (int rc = ck(cudaMemcpyAsync(b->dtiles, b->htiles.data(), b->htiles.size() * sizeof(int4),
                                    cudaMemcpyHostToDevice, st),
                    "batched TTI tile table copy"))
        return rc;
    if (int rc = ck(cudaStreamSynchronize(st), "batched TTI tile table copy")) return rc;
    b->sig = sig;
    return PROP_OK;
}

// a forward-step configuration of every request into the fixed device table
// `slot` (0 or 1), once, before a graph that launches it is captured
int tti_batch_fix(TtiBatch *b, const TtiBatchReq *req, int n, int slot, cudaStream_t st, std::string *err)
{
    auto ck = [&](cudaError_t c, const char *what) {
        if (c == cudaSuccess) return PROP_OK;
        *err = std::string("CUDA error '") + cudaGetErrorString(c) + "' in " + what;
        return c == cudaErrorMemoryAllocation ? PROP_ENOMEM : PROP_ECUDA;
    };
    if (slot < 0) return PROP_EINVAL;
    const int mode = req[0].adjoint ? (req[0].grad ? 2 : 1) : 0;
    for (int i = 0; i < n; i++)
        if (!tti_batchable(req[i].P) || req[i].P->M != req[0].P->M || req[i].adjoint != req[0].adjoint ||
            (req[i].grad != nullptr) != (req[0].grad != nullptr))
            return 1;
    if (int rc = tti_batch_tiles(b, req, n, st, err)) return rc;
    if ((size_t)n > b->fixed_cap) {              // every slot holds n entries
        for (auto &d : b->dfixed) {
            cudaFree(d);
            d = nullptr;
        }
        b->fixed_cap = n;
    }
    if ((size_t)slot >= b->dfixed.size()) {
        b->dfixed.resize(slot + 1, nullptr);
        b->fixed_mode.resize(slot + 1, -1);
    }
    if (!b->dfixed[slot])
        if (int rc = wp_dev_alloc((void **)&b->dfixed[slot], b->fixed_cap * sizeof(TtiShot),
                                  "batched TTI fixed table", err))
            return rc;
    std::vector<TtiShot> H(n);
    int rc = 1;
#define WP_FILL(MM)                                                                                            \
    case MM:                                                                                                   \
        rc = mode == 0 ? tti_batch_fill<MM, 0, 0>(req, n, H.data(), err)                                      \
                       : (mode == 1 ? tti_batch_fill<MM, 1, 0>(req, n, H.data(), err)                         \
                                    : tti_batch_fill<MM, 1, 1>(req, n, H.data(), err));                       \
        break;
    switch (req[0].P->M) {
        WP_FILL(2)
        WP_FILL(4)
        WP_FILL(6)
        WP_FILL(8)
    }
#undef WP_FILL
    if (rc) return rc;
    if (int r2 = ck(cudaMemcpy(b->dfixed[slot], H.data(), n * sizeof(TtiShot), cudaMemcpyHostToDevice),
                    "batched TTI fixed table copy"))
        return r2;
    b->fixed_mode[slot] = mode;
    b->fixed_n = n;
    b->fixed_M = req[0].P->M;
    b->w = req[0].P->w;
    return PROP_OK;
}

// the step of every shot of fixed table `slot` (capturable: launches only)
template <int M, int ADJ, int GRAD>
static int tti_batch_run_fixed(TtiBatch *b, int slot, cudaStream_t st)
{
    const size_t s1 = RL<M>::NS * RL<M>::SZ * sizeof(float) + 64,
                 s2 = NSTAGE * UL<M, ADJ, GRAD>::SZ * sizeof(float) + 64;
    static const bool attr = set_smem(tti_rot_batch<M>, s1) && set_smem(tti_upd_batch<M, ADJ, GRAD>, s2);
    (void)attr;
    const unsigned nt = (unsigned)b->htiles.size();
    const dim3 blk(TZ2, FY + 2, 1);
    tti_rot_batch<M><<<nt, blk, s1, st>>>(b->dfixed[slot], b->dtiles, b->w);
    tti_upd_batch<M, ADJ, GRAD><<<nt, blk, s2, st>>>(b->dfixed[slot], b->dtiles, b->w);
    return cudaGetLastError() == cudaSuccess ? PROP_OK : PROP_ECUDA;
}

int tti_batch_launch_fixed(TtiBatch *b, int slot, cudaStream_t st)
{
    if (slot < 0 || (size_t)slot >= b->dfixed.size() || !b->dfixed[slot]) return PROP_EINVAL;
    const int mode = b->fixed_mode[slot];
#define WP_RUN(MM)                                                                                             \
    case MM:                                                                                                   \
        return mode == 0 ? tti_batch_run_fixed<MM, 0, 0>(b, slot, st)                                         \
                         : (mode == 1 ? tti_batch_run_fixed<MM, 1, 0>(b, slot, st)                            \
                                      : tti_batch_run_fixed<MM, 1, 1>(b, slot, st));
    switch (b->fixed_M) {
        WP_RUN(2)
        WP_RUN(4)
        WP_RUN(6)
        WP_RUN(8)
    }
#undef WP_RUN
    return PROP_EINVAL;
}

int tti_batch_step(TtiBatch *b, const TtiBatchReq *req, int n, cudaStream_t st, std::string *err)
{
    if (n < 1) return PROP_OK;
    const prop_s *P0 = req[0].P;
    const bool grad = req[0].grad != nullptr;
    for (int i = 0; i < n; i++) {
        const prop_s *P = req[i].P;
        if (!tti_batchable(P) || P->M != P0->M || req[i].adjoint != req[0].adjoint ||
            (req[i].grad != nullptr) != grad || (grad && !req[0].adjoint) ||
            memcmp(&P->w, &P0->w, sizeof(FDW)) != 0)
            return 1;
    }
    auto ck = [&](cudaError_t c, const char *what) {
        if (c == cudaSuccess) return PROP_OK;
        *err = std::string("CUDA error '") + cudaGetErrorString(c) + "' in " + what;
        return c == cudaErrorMemoryAllocation ? PROP_ENOMEM : PROP_ECUDA;
    };
    if (int rc = tti_batch_tiles(b, req, n, st, err)) return rc;
    if ((size_t)n > b->shots_cap) {
        cudaFree(b->dshots);
        b->dshots = nullptr;
        b->shots_cap = 0;
        if (int rc = wp_dev_alloc((void **)&b->dshots, n * sizeof(TtiShot), "batched TTI shot table", err)) return rc;
        b->shots_cap = n;
    }
    if ((size_t)n > b->hcap) {
        for (int i = 0; i < TtiBatch::NSLOT; i++) {
            if (b->copied[i]) cudaEventSynchronize(b->copied[i]);
            cudaFreeHost(b->hshots[i]);
            b->hshots[i] = nullptr;
        }
        b->hcap = 0;
        for (int i = 0; i < TtiBatch::NSLOT; i++) {
            if (int rc = ck(cudaMallocHost(&b->hshots[i], n * sizeof(TtiShot)), "batched TTI staging")) return rc;
            if (!b->copied[i])
                if (int rc = ck(cudaEventCreateWithFlags(&b->copied[i], cudaEventDisableTiming),
                                "batched TTI staging event"))
                    return rc;
        }
        b->hcap = n;
    }
    const bool adj = req[0].adjoint;
    switch (P0->M) {
    case 2: return adj ? (grad ? tti_batch_launch<2, 1, 1>(b, req, n, st, err) : tti_batch_launch<2, 1, 0>(b, req, n, st, err))
                       : tti_batch_launch<2, 0, 0>(b, req, n, st, err);
    case 4: return adj ? (grad ? tti_batch_launch<4, 1, 1>(b, req, n, st, err) : tti_batch_launch<4, 1, 0>(b, req, n, st, err))
                       : tti_batch_launch<4, 0, 0>(b, req, n, st, err);
    case 6: return adj ? (grad ? tti_batch_launch<6, 1, 1>(b, req, n, st, err) : tti_batch_launch<6, 1, 0>(b, req, n, st, err))
                       : tti_batch_launch<6, 0, 0>(b, req, n, st, err);
    case 8: return adj ? (grad ? tti_batch_launch<8, 1, 1>(b, req, n, st, err) : tti_batch_launch<8, 1, 0>(b, req, n, st, err))
                       : tti_batch_launch<8, 0, 0>(b, req, n, st, err);
    }
    return 1;
}

bool el_batchable(const prop_s *P) { return P->d.kind == PROP_ELASTIC && tma_usable(P); }

// per-shot entries of one elastic step of every request: mode 0 one table
// H[0..n); mode 1 the three tables of the transposed step with imaging,
// H[0..n) velocity (adjoint), H[n..2n) stress (imaging), H[2n..3n) stress
// (adjoint)
template <int M>
static int el_fill(const ElBatchReq *req, int n, ElShot *H, std::string *err)
{
    const int mode = req[0].mode;
    for (int i = 0; i < n; i++) {
        prop_s *P = req[i].P;
        float *const *S = req[i].S;
        bool ok = true;
        if (mode == 0) {
            ElShot &e = H[i];
            e.g = P->g;
            e.g.dt = req[i].sign * P->g.dt;
            for (int k = 0; k < 9; k++) e.s.f[k] = S[k];
            e.o = F5{};
            ok = vmaps<M>(P, S, S + 3, &e.vm) && tmaps<M>(P, S, S + 3, &e.tm);
            e.xc = P->xchunk;
            e.flag = P->flag;
        } else {
            // the three passes of el_adj_grad: velocity (adjoint), stress
            // (imaging with the forward v^{k+1}), stress (adjoint)
            float *const *sig = P->tmp, *const *w = P->tmp + 6, *const *ep = P->tmp + 9;
            const float *const *v1 = req[i].xk1;
            ElShot &ev = H[i], &e2 = H[n + i], &e1 = H[2 * n + i];
            for (ElShot *e : {&ev, &e2, &e1}) {
                e->g = P->g;
                e->xc = P->xchunk;
                e->flag = P->flag;
                e->o = F5{};
            }
            for (int k = 0; k < 3; k++) {
                ev.s.f[k] = S[k];
                e2.s.f[k] = const_cast<float *>(v1[k]);
                e1.s.f[k] = w[k];
                ev.o.f[k] = w[k];
            }
            for (int k = 0; k < 6; k++) {
                ev.s.f[3 + k] = sig[k];
                e2.s.f[3 + k] = S[3 + k];
                e1.s.f[3 + k] = S[3 + k];
            }
            e2.o = F5{{req[i].g[0], req[i].g[1], ep[0], ep[1], ep[2]}};
            ok = vmaps<M>(P, S, sig, &ev.vm) && tmaps<M>(P, v1, S + 3, &e2.tm) && tmaps<M>(P, w, S + 3, &e1.tm) &&
                 map_of(P, req[i].g[0], FZ, FY, &e2.tm.gl) && map_of(P, req[i].g[1], FZ, FY, &e2.tm.gm);
        }
        if (!ok) {
            *err = "cuTensorMapEncodeTiled failed";
            return PROP_ECUDA;
        }
    }
    return PROP_OK;
}

template <int M>
static int el_batch_launch(TtiBatch *b, const ElBatchReq *req, int n, cudaStream_t st, std::string *err)
{
    auto ck = [&](cudaError_t c, const char *what) {
        if (c == cudaSuccess) return PROP_OK;
        *err = std::string("CUDA error '") + cudaGetErrorString(c) + "' in " + what;
        return c == cudaErrorMemoryAllocation ? PROP_ENOMEM : PROP_ECUDA;
    };
    const int mode = req[0].mode, per = mode == 0 ? 1 : 3;
    const size_t bytes = (size_t)n * per * sizeof(ElShot);
    if (bytes > b->del_cap) {
        cudaFree(b->del);
        b->del = nullptr;
        b->del_cap = 0;
        if (int rc = wp_dev_alloc((void **)&b->del, bytes, "batched elastic shot table", err)) return rc;
        b->del_cap = bytes;
    }
    if (bytes > b->hel_cap) {
        for (int i = 0; i < TtiBatch::NSLOT; i++) {
            if (b->elcopied[i]) cudaEventSynchronize(b->elcopied[i]);
            cudaFreeHost(b->hel[i]);
            b->hel[i] = nullptr;
        }
        b->hel_cap = 0;
        for (int i = 0; i < TtiBatch::NSLOT; i++) {
            if (int rc = ck(cudaMallocHost(&b->hel[i], bytes), "batched elastic staging")) return rc;
            if (!b->elcopied[i])
                if (int rc = ck(cudaEventCreateWithFlags(&b->elcopied[i], cudaEventDisableTiming),
                                "batched elastic staging event"))
                    return rc;
        }
        b->hel_cap = bytes;
    }
    const int slot = (int)(b->calls++ % TtiBatch::NSLOT);
    if (int rc = ck(cudaEventSynchronize(b->elcopied[slot]), "batched elastic staging wait")) return rc;
    ElShot *H = reinterpret_cast<ElShot *>(b->hel[slot]);
    if (int rc = el_fill<M>(req, n, H, err)) return rc;
    if (int rc = ck(cudaMemcpyAsync(b->del, H, bytes, cudaMemcpyHostToDevice, st), "batched elastic table copy"))
        return rc;
    if (int rc = ck(cudaEventRecord(b->elcopied[slot], st), "batched elastic event")) return rc;
    const unsigned nt = (unsigned)b->htiles.size();
    const dim3 blk(TZ2, FY + 2, 1);
    const ElShot *D = reinterpret_cast<const ElShot *>(b->del);
    const FDW &w = req[0].P->w;
    if (mode == 0) {
        const size_t sv = NSTAGE * VL<M>::SZ * sizeof(float) + 64, stt = NSTAGE * TL<M, 0>::SZ * sizeof(float) + 64;
        static const bool attr = set_smem(el_vpass_batch<M, 0>, sv) && set_smem(el_tpass_batch<M, 0>, stt);
        (void)attr;
        el_vpass_batch<M, 0><<<nt, blk, sv, st>>>(D, b->dtiles, w);
        el_tpass_batch<M, 0><<<nt, blk, stt, st>>>(D, b->dtiles, w);
    } else {
        const size_t sv = NSTAGE * VL<M>::SZ * sizeof(float) + 64, s2 = NSTAGE * TL<M, 2>::SZ * sizeof(float) + 64,
                     s1 = NSTAGE * TL<M, 1>::SZ * sizeof(float) + 64;
        static const bool attr = set_smem(el_vpass_batch<M, 1>, sv) && set_smem(el_tpass_batch<M, 2>, s2) &&
                                 set_smem(el_tpass_batch<M, 1>, s1);
        (void)attr;
        for (int i = 0; i < n; i++) el_adj_pre_launch(req[i].P, req[i].S, st);
        el_vpass_batch<M, 1><<<nt, blk, sv, st>>>(D, b->dtiles, w);
        el_tpass_batch<M, 2><<<nt, blk, s2, st>>>(D + n, b->dtiles, w);
        el_tpass_batch<M, 1><<<nt, blk, s1, st>>>(D + 2 * n, b->dtiles, w);
        for (int i = 0; i < n; i++) el_face2_launch(req[i].P, req[i].S, req[i].xk, req[i].xk1, st);
    }
    for (int i = 0; i < n; i++) req[i].P->kern_launches += mode == 0 ? 2 : 3;
    return ck(cudaGetLastError(), "batched elastic step launch");
}

int el_batch_step(TtiBatch *b, const ElBatchReq *req, int n, cudaStream_t st, std::string *err)
{
    if (n < 1) return PROP_OK;
    const prop_s *P0 = req[0].P;
    for (int i = 0; i < n; i++) {
        const prop_s *P = req[i].P;
        if (!el_batchable(P) || P->M != P0->M || req[i].mode != req[0].mode || req[i].sign != req[0].sign)
            return 1;
    }
    std::vector<prop_s *> Ps(n);
    for (int i = 0; i < n; i++) Ps[i] = req[i].P;
    if (int rc = batch_tiles(b, Ps, st, err)) return rc;
    switch (P0->M) {
    case 2: return el_batch_launch<2>(b, req, n, st, err);
    case 4: return el_batch_launch<4>(b, req, n, st, err);
    case 6: return el_batch_launch<6>(b, req, n, st, err);
    case 8: return el_batch_launch<8>(b, req, n, st, err);
    }
    return 1;
}

// fixed table `slot` of an elastic step of every request (mode 0 with sign
// +1: a forward step; mode 1: the transposed step with imaging, three
// tables), for launches that may be captured into a CUDA graph
int el_batch_fix(TtiBatch *b, const ElBatchReq *req, int n, int slot, cudaStream_t st, std::string *err)
{
    auto ck = [&](cudaError_t c, const char *what) {
        if (c == cudaSuccess) return PROP_OK;
        *err = std::string("CUDA error '") + cudaGetErrorString(c) + "' in " + what;
        return c == cudaErrorMemoryAllocation ? PROP_ENOMEM : PROP_ECUDA;
    };
    if (n < 1 || slot < 0) return PROP_EINVAL;
    const prop_s *P0 = req[0].P;
    const int mode = req[0].mode;
    for (int i = 0; i < n; i++)
        if (!el_batchable(req[i].P) || req[i].P->M != P0->M || req[i].mode != mode || (mode == 0 && req[i].sign != 1.f))
            return 1;
    std::vector<prop_s *> Ps(n);
    for (int i = 0; i < n; i++) Ps[i] = req[i].P;
    if (int rc = batch_tiles(b, Ps, st, err)) return rc;
    if ((size_t)n > b->elfixed_cap) {             // every slot holds 3n entries
        for (auto &d : b->elfixed) {
            cudaFree(d);
            d = nullptr;
        }
        b->elfixed_cap = n;
    }
    if ((size_t)slot >= b->elfixed.size()) {
        b->elfixed.resize(slot + 1, nullptr);
        b->elfixed_mode.resize(slot + 1, -1);
    }
    if (!b->elfixed[slot])
        if (int rc = wp_dev_alloc((void **)&b->elfixed[slot], 3 * b->elfixed_cap * sizeof(ElShot),
                                  "batched elastic fixed table", err))
            return rc;
    std::vector<ElShot> H((mode == 0 ? 1 : 3) * n);
    int rc = 1;
    switch (P0->M) {
    case 2: rc = el_fill<2>(req, n, H.data(), err); break;
    case 4: rc = el_fill<4>(req, n, H.data(), err); break;
    case 6: rc = el_fill<6>(req, n, H.data(), err); break;
    case 8: rc = el_fill<8>(req, n, H.data(), err); break;
    }
    if (rc) return rc;
    if (int r2 = ck(cudaMemcpy(b->elfixed[slot], H.data(), H.size() * sizeof(ElShot), cudaMemcpyHostToDevice),
                    "batched elastic fixed table copy"))
        return r2;
    b->elfixed_mode[slot] = mode;
    b->fixed_n = n;
    b->fixed_M = P0->M;
    b->w = P0->w;
    return PROP_OK;
}

template <int M>
static int el_batch_run_fixed(TtiBatch *b, int slot, cudaStream_t st)
{
    const unsigned nt = (unsigned)b->htiles.size();
    const dim3 blk(TZ2, FY + 2, 1);
    const ElShot *D = b->elfixed[slot];
    const int n = b->fixed_n;
    if (b->elfixed_mode[slot] == 0) {
        const size_t sv = NSTAGE * VL<M>::SZ * sizeof(float) + 64, stt = NSTAGE * TL<M, 0>::SZ * sizeof(float) + 64;
        static const bool attr = set_smem(el_vpass_batch<M, 0>, sv) && set_smem(el_tpass_batch<M, 0>, stt);
        (void)attr;
        el_vpass_batch<M, 0><<<nt, blk, sv, st>>>(D, b->dtiles, b->w);
        el_tpass_batch<M, 0><<<nt, blk, stt, st>>>(D, b->dtiles, b->w);
    } else {
        // the three passes only: the pointwise kernels before and after are
        // the caller's (per shot)
        const size_t sv = NSTAGE * VL<M>::SZ * sizeof(float) + 64, s2 = NSTAGE * TL<M, 2>::SZ * sizeof(float) + 64,
                     s1 = NSTAGE * TL<M, 1>::SZ * sizeof(float) + 64;
        static const bool attr = set_smem(el_vpass_batch<M, 1>, sv) && set_smem(el_tpass_batch<M, 2>, s2) &&
                                 set_smem(el_tpass_batch<M, 1>, s1);
        (void)attr;
        el_vpass_batch<M, 1><<<nt, blk, sv, st>>>(D, b->dtiles, b->w);
        el_tpass_batch<M, 2><<<nt, blk, s2, st>>>(D + n, b->dtiles, b->w);
        el_tpass_batch<M, 1><<<nt, blk, s1, st>>>(D + 2 * n, b->dtiles, b->w);
    }
    return cudaGetLastError() == cudaSuccess ? PROP_OK : PROP_ECUDA;
}

// the step of every shot of elastic fixed table `slot` (capturable)
int el_batch_launch_fixed(TtiBatch *b, int slot, cudaStream_t st)
{
    if (slot < 0 || (size_t)slot >= b->elfixed.size() || !b->elfixed[slot]) return PROP_EINVAL;
    switch (b->fixed_M) {
    case 2: return el_batch_run_fixed<2>(b, slot, st);
    case 4: return el_batch_run_fixed<4>(b, slot, st);
    case 6: return el_batch_run_fixed<6>(b, slot, st);
    case 8: return el_batch_run_fixed<8>(b, slot, st);
    }
    return PROP_EINVAL;
}

// centred first derivatives D p, D r and the half-point products
// (D+_i p)(D+_i r) through the TMA rotation pass (see raw_half; NZ a
// multiple of 4)
int tti_raw_half_tma(prop_s *P, const float *p, const float *r, float *const *dp, float *const *dr,
                     float *const *h)
{
    switch (P->M) {
    case 2: return raw_half<2>(P, p, r, dp, dr, h);
    case 4: return raw_half<4>(P, p, r, dp, dr, h);
    case 6: return raw_half<6>(P, p, r, dp, dr, h);
    case 8: return raw_half<8>(P, p, r, dp, dr, h);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
#endif  // WP_TILE_Y == 16
