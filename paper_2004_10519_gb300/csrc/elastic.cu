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

template <int M>
__global__ void __launch_bounds__(TZ *TY)
el_v_kernel(GridDev g, FDW w, Fields9 s, const float *__restrict__ bu, int *flag, int check)
{
    EL_IDX
    float d[3];
    div_tau<M>(g, w, s.f[3], s.f[4], s.f[5], s.f[6], s.f[7], s.f[8], x, y, z, d);
    const float c = g.dt * g.ih;
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float gx = cerjan(g, fx + 0.5f, fy, fz), gy = cerjan(g, fx, fy + 0.5f, fz),
                gz = cerjan(g, fx, fy, fz + 0.5f);
    const float vx = gx * (s.f[0][q] + c * bavg(bu, g, 0, x, y, z) * d[0]);
    const float vy = gy * (s.f[1][q] + c * bavg(bu, g, 1, x, y, z) * d[1]);
    const float vz = gz * (s.f[2][q] + c * bavg(bu, g, 2, x, y, z) * d[2]);
    s.f[0][q] = vx;
    s.f[1][q] = vy;
    s.f[2][q] = vz;
    if (check && !(isfinite(vx) && isfinite(vy) && isfinite(vz))) atomicOr(flag, 1);
}

template <int M>
__global__ void __launch_bounds__(TZ *TY)
el_t_kernel(GridDev g, FDW w, Fields9 s, const float *__restrict__ lam,
            const float *__restrict__ mu, int *flag, int check)
{
    EL_IDX
    float e[6];
    strain<M>(g, w, s.f[0], s.f[1], s.f[2], x, y, z, e);
    const float c = g.dt * g.ih;
    const float l = __ldg(lam + q), m2 = 2.f * __ldg(mu + q);
    const float tr = e[0] + e[1] + e[2];
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float gn = cerjan(g, fx, fy, fz);
    float out[6];
    out[0] = gn * (s.f[3][q] + c * (l * tr + m2 * e[0]));
    out[1] = gn * (s.f[4][q] + c * (l * tr + m2 * e[1]));
    out[2] = gn * (s.f[5][q] + c * (l * tr + m2 * e[2]));
    out[3] = cerjan(g, fx + 0.5f, fy + 0.5f, fz) * (s.f[6][q] + c * muavg(mu, g, 0, 1, x, y, z) * e[3]);
    out[4] = cerjan(g, fx + 0.5f, fy, fz + 0.5f) * (s.f[7][q] + c * muavg(mu, g, 0, 2, x, y, z) * e[4]);
    out[5] = cerjan(g, fx, fy + 0.5f, fz + 0.5f) * (s.f[8][q] + c * muavg(mu, g, 1, 2, x, y, z) * e[5]);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        s.f[3 + i][q] = out[i];
        ok = ok && isfinite(out[i]);
    }
    if (check && !ok) atomicOr(flag, 1);
}

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
    e0[q] = c * s.f[6][q] * e[3];
    e1[q] = c * s.f[7][q] * e[4];
    e2[q] = c * s.f[8][q] * e[5];
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
    f0[q] = c * s.f[0][q] * d[0];
    f1[q] = c * s.f[1][q] * d[1];
    f2[q] = c * s.f[2][q] * d[2];
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

template <int M>
int launch_step(prop_s *P, float *const *S, bool adjoint)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, TY, 1), grd((g.NZ + TZ - 1) / TZ, (g.NY + TY - 1) / TY, g.NX);
    Fields9 s;
    for (int i = 0; i < 9; i++) s.f[i] = S[i];
    prof_begin(P, adjoint ? 3 : 2);
    if (!adjoint) {
        el_v_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, P->bu, P->flag, P->d.check_nan);
        el_t_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, P->lam, P->mu, P->flag,
                                                   P->d.check_nan);
        P->kern_launches += 2;
    } else {
        Fields9 sg;
        for (int i = 0; i < 9; i++) sg.f[i] = P->tmp[i];
        el_adj_pre_kernel<<<grd, blk, 0, P->stream>>>(g, s, sg, P->lam, P->mu);
        el_adj_v_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, sg, P->bu);
        el_adj_t_kernel<M><<<grd, blk, 0, P->stream>>>(g, P->w, s, sg);
        P->kern_launches += 3;
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
    el_grad_gather_kernel<<<grd, blk, 0, P->stream>>>(g, pr[0], pr[1], pr[2], pr[3], pr[4], pr[5],
                                                      gr[1], gr[2]);
    prof_end(P, 4);
    P->kern_launches += 6;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

int el_launch_adj_grad(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1,
                       float *const *g)
{
    switch (P->M) {
    case 2: return launch_adj_grad<2>(P, S, xk, xk1, g);
    case 4: return launch_adj_grad<4>(P, S, xk, xk1, g);
    case 6: return launch_adj_grad<6>(P, S, xk, xk1, g);
    case 8: return launch_adj_grad<8>(P, S, xk, xk1, g);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}

int el_launch_step(prop_s *P, float *const *S, bool adjoint)
{
    switch (P->M) {
    case 2: return launch_step<2>(P, S, adjoint);
    case 4: return launch_step<4>(P, S, adjoint);
    case 6: return launch_step<6>(P, S, adjoint);
    case 8: return launch_step<8>(P, S, adjoint);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
