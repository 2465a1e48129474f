// Elastic velocity-stress kernels (Sec. IV, Eq. elas1, elastic listing).
//
// Staggering: txx,tyy,tzz,lambda,mu,rho at nodes (i,j,k); vx at (i+1/2,j,k),
// vy at (i,j+1/2,k), vz at (i,j,k+1/2); txy at (i+1/2,j+1/2,k), txz at
// (i+1/2,j,k+1/2), tyz at (i,j+1/2,k+1/2); a half index i+1/2 is stored at i.
// Staggered derivatives with zero extension:
//   D+ f (node -> half) at i+1/2 = (1/h) sum_k b_k (f_{i+k}     - f_{i-k+1})
//   D- g (half -> node) at i     = (1/h) sum_k b_k (g_{i+k-1}   - g_{i-k})
// Forward step (listing): v <- g (v + dt b div tau);
//   tau <- g (tau + dt (lambda tr(grad v) I + mu (grad v + grad v^T))) with the
//   new v; buoyancy averaged over the 2 nodes of a face, mu over the 4 nodes
//   of an edge (indices clamped at the grid end).
// Adjoint step (transpose): t = g tbar;  vbar <- g (vbar - dt Dtau(C t));
//   tbar <- t - dt S(b vbar)  (Dtau^T = -S).
#include "common.cuh"

namespace {

constexpr int TZ = 32, TY = 8;

#define EL_IDX                                              \
    const int z = blockIdx.x * TZ + threadIdx.x;            \
    const int y = blockIdx.y * TY + threadIdx.y;            \
    const int x = blockIdx.z;                               \
    if (z >= g.NZ || y >= g.NY) return;                     \
    const long long q = gidx(g, x, y, z);

// staggered derivative sums (without 1/h) at (x,y,z) along axis A
template <int M, int A>
__device__ __forceinline__ float dplus(const float *__restrict__ f, const GridDev &g, const FDW &w,
                                       int x, int y, int z)
{
    float s = 0.f;
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const int a = k, b = -k + 1;
        s += w.b[k - 1] * (ldz(f, g, x + (A == 0) * a, y + (A == 1) * a, z + (A == 2) * a) -
                           ldz(f, g, x + (A == 0) * b, y + (A == 1) * b, z + (A == 2) * b));
    }
    return s;
}
template <int M, int A>
__device__ __forceinline__ float dminus(const float *__restrict__ f, const GridDev &g, const FDW &w,
                                        int x, int y, int z)
{
    float s = 0.f;
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const int a = k - 1, b = -k;
        s += w.b[k - 1] * (ldz(f, g, x + (A == 0) * a, y + (A == 1) * a, z + (A == 2) * a) -
                           ldz(f, g, x + (A == 0) * b, y + (A == 1) * b, z + (A == 2) * b));
    }
    return s;
}

__device__ __forceinline__ float bavg(const float *__restrict__ b, const GridDev &g, int A, int x,
                                      int y, int z)
{
    const int x1 = min(x + (A == 0), g.NX - 1), y1 = min(y + (A == 1), g.NY - 1),
              z1 = min(z + (A == 2), g.NZ - 1);
    return 0.5f * (__ldg(b + gidx(g, x, y, z)) + __ldg(b + gidx(g, x1, y1, z1)));
}
__device__ __forceinline__ float muavg(const float *__restrict__ mu, const GridDev &g, int A1,
                                       int A2, int x, int y, int z)
{
    const int xa = min(x + (A1 == 0), g.NX - 1), ya = min(y + (A1 == 1), g.NY - 1),
              za = min(z + (A1 == 2), g.NZ - 1);
    const int xb = min(x + (A2 == 0), g.NX - 1), yb = min(y + (A2 == 1), g.NY - 1),
              zb = min(z + (A2 == 2), g.NZ - 1);
    const int xc = min(xa + (A2 == 0), g.NX - 1), yc = min(ya + (A2 == 1), g.NY - 1),
              zc = min(za + (A2 == 2), g.NZ - 1);
    return 0.25f * (__ldg(mu + gidx(g, x, y, z)) + __ldg(mu + gidx(g, xa, ya, za)) +
                    __ldg(mu + gidx(g, xb, yb, zb)) + __ldg(mu + gidx(g, xc, yc, zc)));
}

// divergence of stress at the three velocity positions (times h)
template <int M>
__device__ __forceinline__ void div_tau(const GridDev &g, const FDW &w, const float *txx,
                                        const float *tyy, const float *tzz, const float *txy,
                                        const float *txz, const float *tyz, int x, int y, int z,
                                        float *d)
{
    d[0] = dplus<M, 0>(txx, g, w, x, y, z) + dminus<M, 1>(txy, g, w, x, y, z) +
           dminus<M, 2>(txz, g, w, x, y, z);
    d[1] = dminus<M, 0>(txy, g, w, x, y, z) + dplus<M, 1>(tyy, g, w, x, y, z) +
           dminus<M, 2>(tyz, g, w, x, y, z);
    d[2] = dminus<M, 0>(txz, g, w, x, y, z) + dminus<M, 1>(tyz, g, w, x, y, z) +
           dplus<M, 2>(tzz, g, w, x, y, z);
}
// strain-like derivatives of a velocity field (times h):
// e = (D-x vx, D-y vy, D-z vz, D+y vx + D+x vy, D+z vx + D+x vz, D+z vy + D+y vz)
template <int M>
__device__ __forceinline__ void strain(const GridDev &g, const FDW &w, const float *vx,
                                       const float *vy, const float *vz, int x, int y, int z,
                                       float *e)
{
    e[0] = dminus<M, 0>(vx, g, w, x, y, z);
    e[1] = dminus<M, 1>(vy, g, w, x, y, z);
    e[2] = dminus<M, 2>(vz, g, w, x, y, z);
    e[3] = dplus<M, 1>(vx, g, w, x, y, z) + dplus<M, 0>(vy, g, w, x, y, z);
    e[4] = dplus<M, 2>(vx, g, w, x, y, z) + dplus<M, 0>(vz, g, w, x, y, z);
    e[5] = dplus<M, 2>(vy, g, w, x, y, z) + dplus<M, 1>(vz, g, w, x, y, z);
}

struct Fields9 {
    float *f[9];
};

// adjoint pass 1 (pointwise): t = g tbar (in place), sigma = C t -> sg[0..5]
__global__ void __launch_bounds__(TZ *TY)
el_adj_pre_kernel(GridDev g, Fields9 s, Fields9 sg, const float *__restrict__ lam,
                  const float *__restrict__ mu)
{
    EL_IDX
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float gn = cerjan(g, fx, fy, fz);
    const float t0 = gn * s.f[3][q], t1 = gn * s.f[4][q], t2 = gn * s.f[5][q];
    const float t3 = cerjan(g, fx + 0.5f, fy + 0.5f, fz) * s.f[6][q];
    const float t4 = cerjan(g, fx + 0.5f, fy, fz + 0.5f) * s.f[7][q];
    const float t5 = cerjan(g, fx, fy + 0.5f, fz + 0.5f) * s.f[8][q];
    s.f[3][q] = t0; s.f[4][q] = t1; s.f[5][q] = t2;
    s.f[6][q] = t3; s.f[7][q] = t4; s.f[8][q] = t5;
    const float l = __ldg(lam + q), m2 = 2.f * __ldg(mu + q), tr = t0 + t1 + t2;
    sg.f[0][q] = l * tr + m2 * t0;
    sg.f[1][q] = l * tr + m2 * t1;
    sg.f[2][q] = l * tr + m2 * t2;
    sg.f[3][q] = muavg(mu, g, 0, 1, x, y, z) * t3;
    sg.f[4][q] = muavg(mu, g, 0, 2, x, y, z) * t4;
    sg.f[5][q] = muavg(mu, g, 1, 2, x, y, z) * t5;
}

// adjoint pass 2: vbar <- g (vbar - dt Dtau(sigma)); wv = b_avg vbar
template <int M>
__global__ void __launch_bounds__(TZ *TY)
el_adj_v_kernel(GridDev g, FDW w, Fields9 s, Fields9 sg, const float *__restrict__ bu)
{
    EL_IDX
    float d[3];
    div_tau<M>(g, w, sg.f[0], sg.f[1], sg.f[2], sg.f[3], sg.f[4], sg.f[5], x, y, z, d);
    const float c = g.dt * g.ih;
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float vx = cerjan(g, fx + 0.5f, fy, fz) * (s.f[0][q] - c * d[0]);
    const float vy = cerjan(g, fx, fy + 0.5f, fz) * (s.f[1][q] - c * d[1]);
    const float vz = cerjan(g, fx, fy, fz + 0.5f) * (s.f[2][q] - c * d[2]);
    s.f[0][q] = vx;
    s.f[1][q] = vy;
    s.f[2][q] = vz;
    sg.f[6][q] = bavg(bu, g, 0, x, y, z) * vx;
    sg.f[7][q] = bavg(bu, g, 1, x, y, z) * vy;
    sg.f[8][q] = bavg(bu, g, 2, x, y, z) * vz;
}

// adjoint pass 3: tbar <- t - dt S(wv)
template <int M>
__global__ void __launch_bounds__(TZ *TY)
el_adj_t_kernel(GridDev g, FDW w, Fields9 s, Fields9 sg)
{
    EL_IDX
    float e[6];
    strain<M>(g, w, sg.f[6], sg.f[7], sg.f[8], x, y, z, e);
    const float c = g.dt * g.ih;
#pragma unroll
    for (int i = 0; i < 6; i++) s.f[3 + i][q] -= c * e[i];
}

// ---- gradient of one forward step k (X^k -> X^{k+1}) --------------------
// t = g tbar^{k+1} (already tapered in place by el_adj_pre_kernel), strain of
// the forward v^{k+1}:  g_lam += dt tr(t_d) tr(e);  g_mu += 2 dt sum t_ii e_ii;
// edge products ep_c = dt t_c e_c (c = xy, xz, yz), scattered 1/4 to nodes.
template <int M>
__global__ void __launch_bounds__(TZ *TY)
el_grad_lm_kernel(GridDev g, FDW w, Fields9 s, Fields9 xf1, float *__restrict__ glam,
                  float *__restrict__ gmu, float *__restrict__ e0, float *__restrict__ e1,
                  float *__restrict__ e2)
{
    EL_IDX
    float e[6];
    strain<M>(g, w, xf1.f[0], xf1.f[1], xf1.f[2], x, y, z, e);
    const float c = g.dt * g.ih;
    const float t0 = s.f[3][q], t1 = s.f[4][q], t2 = s.f[5][q];
    glam[q] += c * (t0 + t1 + t2) * (e[0] + e[1] + e[2]);
    gmu[q] += 2.f * c * (t0 * e[0] + t1 * e[1] + t2 * e[2]);
    e0[q] += c * s.f[6][q] * e[3];
    e1[q] += c * s.f[7][q] * e[4];
    e2[q] += c * s.f[8][q] * e[5];
}
// face products fp_c = dt vbar^k_c (Dtau tau^k)_c (c = x, y, z), scattered 1/2
template <int M>
__global__ void __launch_bounds__(TZ *TY)
el_grad_b_kernel(GridDev g, FDW w, Fields9 s, Fields9 xf0, float *__restrict__ f0,
                 float *__restrict__ f1, float *__restrict__ f2)
{
    EL_IDX
    float d[3];
    div_tau<M>(g, w, xf0.f[3], xf0.f[4], xf0.f[5], xf0.f[6], xf0.f[7], xf0.f[8], x, y, z, d);
    const float c = g.dt * g.ih;
    f0[q] += c * s.f[0][q] * d[0];
    f1[q] += c * s.f[1][q] * d[1];
    f2[q] += c * s.f[2][q] * d[2];
}

// Face products of the b-gradient without a stencil.  The forward velocity
// update v^{k+1} = g (v^k + (dt/h) b_avg Dtau(tau^k)) gives
// (dt/h) Dtau(tau^k) = (v^{k+1}/g - v^k) / b_avg at each velocity point, so
// fp_c = vbar_c (v^{k+1}_c / g_c - v^k_c) / b_avg,c equals the product of
// el_grad_b_kernel.  Two z points per thread, 8-byte accesses (NZ even, as
// on the TMA path that uses it); tapers and averages as in the TMA passes.
__global__ void __launch_bounds__(256)
el_face2_kernel(GridDev g, Fields9 s, Fields9 xf0, Fields9 xf1, const float *__restrict__ bu,
                float *__restrict__ f0, float *__restrict__ f1, float *__restrict__ f2)
{
    const int x = blockIdx.z, y = blockIdx.y * 8 + threadIdx.y, z = 2 * (blockIdx.x * 32 + threadIdx.x);
    if (y >= g.NY || z >= g.NZ) return;
    const long long pl = (long long)g.NY * g.NZ, q = ((long long)x * g.NY + y) * g.NZ + z;
    auto ld = [](const float *p, long long o) { return __ldg(reinterpret_cast<const float2 *>(p + o)); };
    // accumulate into the face-product sums (read before written, own points only)
    auto st = [](float *p, long long o, float a, float b) {
        float2 *d = reinterpret_cast<float2 *>(p + o);
        const float2 v = *d;
        *d = make_float2(v.x + a, v.y + b);
    };
    const float2 b0 = ld(bu, q);
    const float2 bX = x + 1 < g.NX ? ld(bu, q + pl) : b0, bY = y + 1 < g.NY ? ld(bu, q + g.NZ) : b0;
    const float bz2 = z + 2 < g.NZ ? __ldg(bu + q + 2) : b0.y;
    const float *tz = g.tab + 2 * (g.NX + g.NY);
    const float gxn = __ldg(g.tab + 2 * x), gxh = __ldg(g.tab + 2 * x + 1);
    const float gyn = __ldg(g.tab + 2 * g.NX + 2 * y), gyh = __ldg(g.tab + 2 * g.NX + 2 * y + 1);
    const float gzn0 = __ldg(tz + 2 * z), gzh0 = __ldg(tz + 2 * z + 1);
    const float gzn1 = __ldg(tz + 2 * z + 2), gzh1 = __ldg(tz + 2 * z + 3);
    const float2 u0 = ld(s.f[0], q), u1 = ld(s.f[1], q), u2 = ld(s.f[2], q);
    const float2 a0 = ld(xf0.f[0], q), a1 = ld(xf0.f[1], q), a2 = ld(xf0.f[2], q);
    const float2 c0 = ld(xf1.f[0], q), c1 = ld(xf1.f[1], q), c2 = ld(xf1.f[2], q);
    st(f0, q, u0.x * (c0.x / (gxh * gyn * gzn0) - a0.x) / (0.5f * (b0.x + bX.x)),
       u0.y * (c0.y / (gxh * gyn * gzn1) - a0.y) / (0.5f * (b0.y + bX.y)));
    st(f1, q, u1.x * (c1.x / (gxn * gyh * gzn0) - a1.x) / (0.5f * (b0.x + bY.x)),
       u1.y * (c1.y / (gxn * gyh * gzn1) - a1.y) / (0.5f * (b0.y + bY.y)));
    st(f2, q, u2.x * (c2.x / (gxn * gyn * gzh0) - a2.x) / (0.5f * (b0.x + b0.y)),
       u2.y * (c2.y / (gxn * gyn * gzh1) - a2.y) / (0.5f * (b0.y + bz2)));
}

// gather of the scattered products: a node receives 1/4 of each of the 4
// edges around it in each plane (clamped averaging transposed) and 1/2 of
// the 2 faces along each axis.
__device__ __forceinline__ float gather_edge(const float *__restrict__ e, const GridDev &g, int A1,
                                             int A2, int x, int y, int z)
{
    // edge (x', y') uses nodes x', min(x'+1, n-1) along A1 (same for A2)
    int c1 = A1 == 0 ? x : (A1 == 1 ? y : z), n1 = A1 == 0 ? g.NX : (A1 == 1 ? g.NY : g.NZ);
    int c2 = A2 == 0 ? x : (A2 == 1 ? y : z), n2 = A2 == 0 ? g.NX : (A2 == 1 ? g.NY : g.NZ);
    // node c receives from edge c (twice at c = n-1, where the clamped second
    // node coincides with the first) and from edge c-1
    float s = 0.f;
    for (int a = 0; a < 2; a++) {
        const int e1 = c1 - a;
        if (e1 < 0) continue;
        const float w1 = (a == 0 && c1 == n1 - 1) ? 2.f : 1.f;
        for (int b = 0; b < 2; b++) {
            const int e2 = c2 - b;
            if (e2 < 0) continue;
            const float w2 = (b == 0 && c2 == n2 - 1) ? 2.f : 1.f;
            int ex = x, ey = y, ez = z;
            if (A1 == 0) ex = e1; else if (A1 == 1) ey = e1; else ez = e1;
            if (A2 == 0) ex = e2; else if (A2 == 1) ey = e2; else ez = e2;
            s += w1 * w2 * e[gidx(g, ex, ey, ez)];
        }
    }
    return 0.25f * s;
}

__global__ void __launch_bounds__(TZ *TY)
el_grad_gather_kernel(GridDev g, const float *__restrict__ ep0, const float *__restrict__ ep1,
                      const float *__restrict__ ep2, const float *__restrict__ fp0,
                      const float *__restrict__ fp1, const float *__restrict__ fp2,
                      float *__restrict__ gmu, float *__restrict__ gb)
{
    EL_IDX
    gmu[q] += gather_edge(ep0, g, 0, 1, x, y, z) + gather_edge(ep1, g, 0, 2, x, y, z) +
              gather_edge(ep2, g, 1, 2, x, y, z);
    float s = 0.f;
    const float *fp[3] = {fp0, fp1, fp2};
    const int c[3] = {x, y, z}, n[3] = {g.NX, g.NY, g.NZ};
    for (int A = 0; A < 3; A++) {
        // face i maps to nodes i and min(i+1, n-1)
        s += fp[A][q] * (c[A] == n[A] - 1 ? 2.f : 1.f);
        if (c[A] >= 1) {
            int xx = x - (A == 0), yy = y - (A == 1), zz = z - (A == 2);
            s += fp[A][gidx(g, xx, yy, zz)];
        }
    }
    gb[q] += 0.5f * s;
}

// ---------------------------------------------------------------------------
// Tiled transposed passes (tbar form, used by prop_step's adjoint).  A CTA
// owns an FZ x FY tile of (y, z) columns and streams along x over a chunk of
// planes.  x-derivatives come from per-thread register queues (2M values),
// y/z-derivatives from shared-memory planes with an M-point halo; values
// outside the grid read as 0.
// ---------------------------------------------------------------------------
constexpr int FZ = 32, FY = 16, FT = FZ * FY;

// taper of one staggered position from the per-axis tables
WP_DEV float tp(const GridDev &g, int x, int hx, int y, int hy, int z, int hz)
{
    return __ldg(g.tab + 2 * x + hx) * __ldg(g.tab + 2 * g.NX + 2 * y + hy) *
           __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * z + hz);
}

// ---- tiled adjoint passes -------------------------------------------------
// C (g tbar) at a node, diagonal component c (0..2); 0 outside the grid
WP_DEV float adj_sdiag(const GridDev &g, const Fields9 &s, const float *__restrict__ lam,
                       const float *__restrict__ mu, int c, int x, int y, int z)
{
    if (!(x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ)) return 0.f;
    const long long q = gidx(g, x, y, z);
    const float gn = tp(g, x, 0, y, 0, z, 0);
    const float t0 = gn * s.f[3][q], t1 = gn * s.f[4][q], t2 = gn * s.f[5][q];
    const float tc = c == 0 ? t0 : (c == 1 ? t1 : t2);
    return __ldg(lam + q) * (t0 + t1 + t2) + 2.f * __ldg(mu + q) * tc;
}
// C (g tbar) on an edge: mu averaged over the 4 nodes of the (A1, A2) plane
template <int A1, int A2>
WP_DEV float adj_sedge(const GridDev &g, const float *tc, const float *__restrict__ mu, int x,
                       int y, int z)
{
    if (!(x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ)) return 0.f;
    const long long q = gidx(g, x, y, z);
    const long long d1 = A1 == 0 ? (x + 1 < g.NX ? (long long)g.NY * g.NZ : 0)
                                 : (y + 1 < g.NY ? (long long)g.NZ : 0);
    const long long d2 = A2 == 1 ? (y + 1 < g.NY ? (long long)g.NZ : 0) : (z + 1 < g.NZ ? 1 : 0);
    const float mavg = 0.25f * (__ldg(mu + q) + __ldg(mu + q + d1) + __ldg(mu + q + d2) +
                                __ldg(mu + q + d1 + d2));
    const float gt = tp(g, x, A1 == 0, y, (A1 == 1) || (A2 == 1), z, A2 == 2);
    return mavg * gt * tc[q];
}
// b_avg * vbar at a velocity point of component c; 0 outside the grid
WP_DEV float adj_bv(const GridDev &g, const float *__restrict__ v, const float *__restrict__ bu, int c,
                    int x, int y, int z)
{
    if (!(x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ)) return 0.f;
    const long long q = gidx(g, x, y, z);
    long long d = 0;
    if (c == 0) d = x + 1 < g.NX ? (long long)g.NY * g.NZ : 0;
    else if (c == 1) d = y + 1 < g.NY ? (long long)g.NZ : 0;
    else d = z + 1 < g.NZ ? 1 : 0;
    return 0.5f * (__ldg(bu + q) + __ldg(bu + q + d)) * v[q];
}

// adjoint velocity pass: vbar <- g (vbar - dt Dtau(C g tbar))
template <int M>
__global__ void __launch_bounds__(FT, 2)
el_adj_v_tiled(GridDev g, FDW w, Fields9 s, const float *__restrict__ lam,
               const float *__restrict__ mu, int xc)
{
    constexpr int HY = FY + 2 * M, HZ = FZ + 2 * M, Q = 2 * M;
    __shared__ float s_xy[HY][FZ], s_yy[HY][FZ], s_yz[HY][HZ], s_xz[FY][HZ], s_zz[FY][HZ];
    const int tz = threadIdx.x, ty = threadIdx.y;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    const float *txy = s.f[6], *txz = s.f[7], *tyz = s.f[8];
    float qxx[Q], qxy[Q], qxz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qxx[j] = adj_sdiag(g, s, lam, mu, 0, xa - M + 1 + j, y, z);
        qxy[j] = adj_sedge<0, 1>(g, txy, mu, xa - M + j, y, z);
        qxz[j] = adj_sedge<0, 2>(g, txz, mu, xa - M + j, y, z);
    }
    const bool act = y < g.NY && z < g.NZ;
    const float c = g.dt * g.ih;
    for (int x = xa; x < xb; x++) {
        qxx[Q - 1] = adj_sdiag(g, s, lam, mu, 0, x + M, y, z);
        qxy[Q - 1] = adj_sedge<0, 1>(g, txy, mu, x + M - 1, y, z);
        qxz[Q - 1] = adj_sedge<0, 2>(g, txz, mu, x + M - 1, y, z);
        __syncthreads();
        s_xy[ty + M][tz] = qxy[M];
        s_xz[ty][tz + M] = qxz[M];
        s_yy[ty + M][tz] = adj_sdiag(g, s, lam, mu, 1, x, y, z);
        s_zz[ty][tz + M] = adj_sdiag(g, s, lam, mu, 2, x, y, z);
        s_yz[ty + M][tz + M] = adj_sedge<1, 2>(g, tyz, mu, x, y, z);
        if (ty < M) {
            const int ya = y0 - M + ty, yb = y0 + FY + ty;
            s_xy[ty][tz] = adj_sedge<0, 1>(g, txy, mu, x, ya, z);
            s_yy[ty][tz] = adj_sdiag(g, s, lam, mu, 1, x, ya, z);
            s_yz[ty][tz + M] = adj_sedge<1, 2>(g, tyz, mu, x, ya, z);
            s_xy[ty + FY + M][tz] = adj_sedge<0, 1>(g, txy, mu, x, yb, z);
            s_yy[ty + FY + M][tz] = adj_sdiag(g, s, lam, mu, 1, x, yb, z);
            s_yz[ty + FY + M][tz + M] = adj_sedge<1, 2>(g, tyz, mu, x, yb, z);
        }
        if (tz < M) {
            const int za = z0 - M + tz, zb = z0 + FZ + tz;
            s_xz[ty][tz] = adj_sedge<0, 2>(g, txz, mu, x, y, za);
            s_zz[ty][tz] = adj_sdiag(g, s, lam, mu, 2, x, y, za);
            s_yz[ty + M][tz] = adj_sedge<1, 2>(g, tyz, mu, x, y, za);
            s_xz[ty][tz + FZ + M] = adj_sedge<0, 2>(g, txz, mu, x, y, zb);
            s_zz[ty][tz + FZ + M] = adj_sdiag(g, s, lam, mu, 2, x, y, zb);
            s_yz[ty + M][tz + FZ + M] = adj_sedge<1, 2>(g, tyz, mu, x, y, zb);
        }
        __syncthreads();
        if (act) {
            float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float b = w.b[k - 1];
                d0 += b * ((qxx[M - 1 + k] - qxx[M - k]) +
                           (s_xy[ty + M + k - 1][tz] - s_xy[ty + M - k][tz]) +
                           (s_xz[ty][tz + M + k - 1] - s_xz[ty][tz + M - k]));
                d1 += b * ((qxy[M + k - 1] - qxy[M - k]) +
                           (s_yy[ty + M + k][tz] - s_yy[ty + M - k + 1][tz]) +
                           (s_yz[ty + M][tz + M + k - 1] - s_yz[ty + M][tz + M - k]));
                d2 += b * ((qxz[M + k - 1] - qxz[M - k]) +
                           (s_yz[ty + M + k - 1][tz + M] - s_yz[ty + M - k][tz + M]) +
                           (s_zz[ty][tz + M + k] - s_zz[ty][tz + M - k + 1]));
            }
            const long long q = gidx(g, x, y, z);
            s.f[0][q] = tp(g, x, 1, y, 0, z, 0) * (s.f[0][q] - c * d0);
            s.f[1][q] = tp(g, x, 0, y, 1, z, 0) * (s.f[1][q] - c * d1);
            s.f[2][q] = tp(g, x, 0, y, 0, z, 1) * (s.f[2][q] - c * d2);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qxx[j] = qxx[j + 1];
            qxy[j] = qxy[j + 1];
            qxz[j] = qxz[j + 1];
        }
    }
}

// adjoint stress pass: tbar <- g tbar - dt S(b_avg vbar)
template <int M>
__global__ void __launch_bounds__(FT, 2)
el_adj_t_tiled(GridDev g, FDW w, Fields9 s, const float *__restrict__ bu, int xc)
{
    constexpr int HY = FY + 2 * M, HZ = FZ + 2 * M, Q = 2 * M;
    __shared__ float s_vx[HY][HZ], s_vy[HY][HZ], s_vz[HY][HZ];
    const int tz = threadIdx.x, ty = threadIdx.y;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    const float *vxp = s.f[0], *vyp = s.f[1], *vzp = s.f[2];
    float qvx[Q], qvy[Q], qvz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qvx[j] = adj_bv(g, vxp, bu, 0, xa - M + j, y, z);
        qvy[j] = adj_bv(g, vyp, bu, 1, xa - M + 1 + j, y, z);
        qvz[j] = adj_bv(g, vzp, bu, 2, xa - M + 1 + j, y, z);
    }
    const bool act = y < g.NY && z < g.NZ;
    const float c = g.dt * g.ih;
    for (int x = xa; x < xb; x++) {
        qvx[Q - 1] = adj_bv(g, vxp, bu, 0, x + M - 1, y, z);
        qvy[Q - 1] = adj_bv(g, vyp, bu, 1, x + M, y, z);
        qvz[Q - 1] = adj_bv(g, vzp, bu, 2, x + M, y, z);
        __syncthreads();
        s_vx[ty + M][tz + M] = qvx[M];
        s_vy[ty + M][tz + M] = qvy[M - 1];
        s_vz[ty + M][tz + M] = qvz[M - 1];
        if (ty < M) {
            const int ya = y0 - M + ty, yb = y0 + FY + ty;
            s_vx[ty][tz + M] = adj_bv(g, vxp, bu, 0, x, ya, z);
            s_vy[ty][tz + M] = adj_bv(g, vyp, bu, 1, x, ya, z);
            s_vz[ty][tz + M] = adj_bv(g, vzp, bu, 2, x, ya, z);
            s_vx[ty + FY + M][tz + M] = adj_bv(g, vxp, bu, 0, x, yb, z);
            s_vy[ty + FY + M][tz + M] = adj_bv(g, vyp, bu, 1, x, yb, z);
            s_vz[ty + FY + M][tz + M] = adj_bv(g, vzp, bu, 2, x, yb, z);
        }
        if (tz < M) {
            const int za = z0 - M + tz, zb = z0 + FZ + tz;
            s_vx[ty + M][tz] = adj_bv(g, vxp, bu, 0, x, y, za);
            s_vy[ty + M][tz] = adj_bv(g, vyp, bu, 1, x, y, za);
            s_vz[ty + M][tz] = adj_bv(g, vzp, bu, 2, x, y, za);
            s_vx[ty + M][tz + FZ + M] = adj_bv(g, vxp, bu, 0, x, y, zb);
            s_vy[ty + M][tz + FZ + M] = adj_bv(g, vyp, bu, 1, x, y, zb);
            s_vz[ty + M][tz + FZ + M] = adj_bv(g, vzp, bu, 2, x, y, zb);
        }
        __syncthreads();
        if (act) {
            float exx = 0.f, eyy = 0.f, ezz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
            const int cy = ty + M, cz = tz + M;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float b = w.b[k - 1];
                exx += b * (qvx[M + k - 1] - qvx[M - k]);
                eyy += b * (s_vy[cy + k - 1][cz] - s_vy[cy - k][cz]);
                ezz += b * (s_vz[cy][cz + k - 1] - s_vz[cy][cz - k]);
                gxy += b * ((s_vx[cy + k][cz] - s_vx[cy - k + 1][cz]) + (qvy[M - 1 + k] - qvy[M - k]));
                gxz += b * ((s_vx[cy][cz + k] - s_vx[cy][cz - k + 1]) + (qvz[M - 1 + k] - qvz[M - k]));
                gyz += b * ((s_vy[cy][cz + k] - s_vy[cy][cz - k + 1]) + (s_vz[cy + k][cz] - s_vz[cy - k + 1][cz]));
            }
            const long long q = gidx(g, x, y, z);
            const float gn = tp(g, x, 0, y, 0, z, 0);
            s.f[3][q] = gn * s.f[3][q] - c * exx;
            s.f[4][q] = gn * s.f[4][q] - c * eyy;
            s.f[5][q] = gn * s.f[5][q] - c * ezz;
            s.f[6][q] = tp(g, x, 1, y, 1, z, 0) * s.f[6][q] - c * gxy;
            s.f[7][q] = tp(g, x, 1, y, 0, z, 1) * s.f[7][q] - c * gxz;
            s.f[8][q] = tp(g, x, 0, y, 1, z, 1) * s.f[8][q] - c * gyz;
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qvx[j] = qvx[j + 1];
            qvy[j] = qvy[j + 1];
            qvz[j] = qvz[j + 1];
        }
    }
}

template <int M>
int launch_step(prop_s *P, float *const *S, bool adjoint)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, g.NX);
    Fields9 s;
    for (int i = 0; i < 9; i++) s.f[i] = S[i];
    if (!adjoint) return tma_usable(P) ? el_launch_tma(P, S, 1.f) : el_launch_fast(P, S, 1.f);
    prof_begin(P, 3);
    {
        const int xc = P->xchunk;
        dim3 fb(FZ, FY, 1), fg((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
        el_adj_v_tiled<M><<<fg, fb, 0, P->stream>>>(g, P->w, s, P->lam, P->mu, xc);
        el_adj_t_tiled<M><<<fg, fb, 0, P->stream>>>(g, P->w, s, P->bu, xc);
        P->kern_launches += 2;
    }
    prof_end(P, adjoint ? 3 : 2);
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

template <int M>
int launch_adj_grad(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1,
                    float *const *gr)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, g.NX);
    Fields9 s, sg, f0, f1;
    for (int i = 0; i < 9; i++) {
        s.f[i] = S[i];
        sg.f[i] = P->tmp[i];
        f0.f[i] = const_cast<float *>(xk[i]);
        f1.f[i] = const_cast<float *>(xk1[i]);
    }
    float *const *pr = P->tmp + 9;   // 6 product arrays
    prof_begin(P, 4);
    el_adj_pre_kernel<<<grd, blk, 0, P->stream>>>(g, s, sg, P->lam, P->mu);
    el_grad_lm_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, f1, gr[0], gr[1], pr[0], pr[1], pr[2]);
    el_adj_v_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, sg, P->bu);
    el_grad_b_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, f0, pr[3], pr[4], pr[5]);
    el_adj_t_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, sg);
    prof_end(P, 4);
    P->kern_launches += 5;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

// the same transposed step with imaging on the TMA-fed passes: pointwise
// tapering and stiffness, three streaming passes (velocity, imaging, stress;
// stencil_tma.cu), pointwise face products, gather
int launch_adj_grad_tma(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1,
                        float *const *gr)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, g.NX);
    Fields9 s, sg, f0, f1;
    for (int i = 0; i < 9; i++) {
        s.f[i] = S[i];
        sg.f[i] = P->tmp[i];
        f0.f[i] = const_cast<float *>(xk[i]);
        f1.f[i] = const_cast<float *>(xk1[i]);
    }
    float *const *pr = P->tmp + 9;   // edge products pr[0..2], face products pr[3..5]
    prof_begin(P, 4);
    el_adj_pre_kernel<<<grd, blk, 0, P->stream>>>(g, s, sg, P->lam, P->mu);
    WP_TRY(el_adj_grad_tma(P, S, P->tmp, P->tmp + 6, xk1, gr, pr));
    el_face2_kernel<<<dim3((g.NZ + 63) / 64, (g.NY + 7) / 8, g.NX), dim3(32, 8, 1), 0, P->stream>>>(
        g, s, f0, f1, P->bu, pr[3], pr[4], pr[5]);
    prof_end(P, 4);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// the pointwise kernels before and after the three TMA passes of a
// transposed step with imaging, on a given stream (batched shots: the
// passes are shared, these run per shot)
void el_adj_pre_launch(prop_s *P, float *const *S, cudaStream_t st)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, g.NX);
    Fields9 s, sg;
    for (int i = 0; i < 9; i++) {
        s.f[i] = S[i];
        sg.f[i] = P->tmp[i];
    }
    el_adj_pre_kernel<<<grd, blk, 0, st>>>(g, s, sg, P->lam, P->mu);
    P->kern_launches += 1;
}

void el_face2_launch(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1, cudaStream_t st)
{
    const GridDev &g = P->g;
    Fields9 s, f0, f1;
    for (int i = 0; i < 9; i++) {
        s.f[i] = S[i];
        f0.f[i] = const_cast<float *>(xk[i]);
        f1.f[i] = const_cast<float *>(xk1[i]);
    }
    float *const *pr = P->tmp + 9;
    el_face2_kernel<<<dim3((g.NZ + 63) / 64, (g.NY + 7) / 8, g.NX), dim3(32, 8, 1), 0, st>>>(
        g, s, f0, f1, P->bu, pr[3], pr[4], pr[5]);
    P->kern_launches += 1;
}

// the edge and face products are summed over the steps of a sweep in
// tmp[9..14] (the averaging transposes are linear and the same every step)
// and gathered onto the nodes once at the end
int el_grad_gather(prop_s *P, float *const *g)
{
    const GridDev &gd = P->g;
    dim3 blk(TZ, TY, 1), grd((gd.NZ + TZ - 1) / TZ, (gd.NY + TY - 1) / TY, gd.NX);
    float *const *pr = P->tmp + 9;
    el_grad_gather_kernel<<<grd, blk, 0, P->stream>>>(gd, pr[0], pr[1], pr[2], pr[3], pr[4], pr[5], g[1], g[2]);
    P->kern_launches += 1;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

int el_launch_adj_grad(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1,
                       float *const *g)
{
    if (P->rdv && el_batchable(P)) {
        ElBatchReq r{P, {}, 1, 1.f, {}, {}, {g[0], g[1], g[2]}};
        for (int i = 0; i < 9; i++) {
            r.S[i] = S[i];
            r.xk[i] = xk[i];
            r.xk1[i] = xk1[i];
        }
        return rdv_el_step(P, r);
    }
    if (tma_usable(P)) return launch_adj_grad_tma(P, S, xk, xk1, g);
    switch (P->M) {
    case 2: return launch_adj_grad<2>(P, S, xk, xk1, g);
    case 4: return launch_adj_grad<4>(P, S, xk, xk1, g);
    case 6: return launch_adj_grad<6>(P, S, xk, xk1, g);
    case 8: return launch_adj_grad<8>(P, S, xk, xk1, g);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

int el_step_adjoint_u(prop_s *P, float *const *S)
{
    if (P->rdv && el_batchable(P)) {
        ElBatchReq r{P, {}, 0, -1.f, {}, {}, {}};
        for (int i = 0; i < 9; i++) r.S[i] = S[i];
        return rdv_el_step(P, r);
    }
    return tma_usable(P) ? el_launch_tma(P, S, -1.f) : el_launch_fast(P, S, -1.f);
}

int el_launch_step(prop_s *P, float *const *S, bool adjoint)
{
    if (!adjoint && P->rdv && el_batchable(P)) {
        ElBatchReq r{P, {}, 0, 1.f, {}, {}, {}};
        for (int i = 0; i < 9; i++) r.S[i] = S[i];
        return rdv_el_step(P, r);
    }
    switch (P->M) {
    case 2: return launch_step<2>(P, S, adjoint);
    case 4: return launch_step<4>(P, S, adjoint);
    case 6: return launch_step<6>(P, S, adjoint);
    case 8: return launch_step<8>(P, S, adjoint);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
