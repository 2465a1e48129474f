// Isotropic acoustic propagator (Sec. II-A, Eq. acou; m u_tt - laplace(u) +
// damp u_t = q of the wave-equation listing), second-order leapfrog with the
// damping layer of the TTI path:
//   u^{n+1} = (dt^2 L u^n + 2 m u^n - B u^{n-1}) / A,  A, B = m (1 +- sig dt/2),
// L = sum over axes of the centred second derivative of the space order.
// L is symmetric, so the transposed step is the same map.  The TMA-fed pass
// (stencil_tma.cu) runs when NZ % 4 == 0; this file holds the dispatch and
// a direct-load kernel for any NZ.
#include "tile.cuh"

namespace {

using tile::lz;

// one point per thread; grid (ceil(NZ/32), ceil(NY/8), NX)
template <int M, int GRAD>
__global__ void __launch_bounds__(256)
acu_direct(GridDev g, FDW w, const float *__restrict__ u1, float *u0, const float *__restrict__ m,
           const float *__restrict__ uf, float *grad, int *flag, int check)
{
    const int z = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, x = blockIdx.z;
    if (z >= g.NZ || y >= g.NY) return;
    const long long q = gidx(g, x, y, z);
    float lap = 3.f * w.d2[0] * u1[q];
#pragma unroll
    for (int k = 1; k <= M; k++)
        lap += w.d2[k] * ((lz(u1, g, x + k, y, z) + lz(u1, g, x - k, y, z)) +
                          (lz(u1, g, x, y + k, z) + lz(u1, g, x, y - k, z)) +
                          (lz(u1, g, x, y, z + k) + lz(u1, g, x, y, z - k)));
    lap *= g.ih * g.ih;
    const float dt2 = g.dt * g.dt;
    const float sd = 0.5f * g.dt * (__ldg(g.tab + x) + __ldg(g.tab + g.NX + y) + __ldg(g.tab + g.NX + g.NY + z));
    const float mm = m[q], A = mm * (1.f + sd), Bc = mm * (1.f - sd);
    const float un = (dt2 * lap + 2.f * mm * u1[q] - Bc * u0[q]) / A;
    u0[q] = un;
    if (GRAD) grad[q] -= dt2 * uf[q] * lap / mm;
    if (check && !isfinite(un)) atomicOr(flag, 1);
}

template <int M>
int launch_direct(prop_s *P, float *const *S, const float *uf, float *grad)
{
    const GridDev &g = P->g;
    dim3 blk(32, 8), grd((g.NZ + 31) / 32, (g.NY + 7) / 8, g.NX);
    if (grad)
        acu_direct<M, 1><<<grd, blk, 0, P->stream>>>(g, P->w, S[0], S[1], P->m, uf, grad, P->flag, P->d.check_nan);
    else
        acu_direct<M, 0><<<grd, blk, 0, P->stream>>>(g, P->w, S[0], S[1], P->m, uf, grad, P->flag,
                                                     P->d.check_nan);
    P->kern_launches += 1;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// one acoustic step of state S (S[0] = u^n, S[1] = u^{n-1}, overwritten by
// u^{n+1}); grad != NULL: transposed step with imaging against uf
int acu_launch_step(prop_s *P, float *const *S, const float *uf, float *grad)
{
    if (tma_usable(P)) return acu_launch_tma(P, S, uf, grad);
    const int id = grad ? 7 : 6;
    prof_begin(P, id);
    int rc;
    switch (P->M) {
    case 2: rc = launch_direct<2>(P, S, uf, grad); break;
    case 4: rc = launch_direct<4>(P, S, uf, grad); break;
    case 6: rc = launch_direct<6>(P, S, uf, grad); break;
    case 8: rc = launch_direct<8>(P, S, uf, grad); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, id);
    return rc;
}
