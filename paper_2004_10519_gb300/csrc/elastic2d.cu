// 2D elastic propagator (x-z plane): the velocity-stress system of Sec. IV-A
// (Eq. elas1, elastic listing) with every y term dropped, as in the 2D
// example of Sec. IV-B.  Fields on the staggered grid of the 3D system:
// vx at (x+1/2, z), vz at (x, z+1/2), txx and tzz at nodes, txz at
// (x+1/2, z+1/2); b averaged over the two nodes of a velocity point, mu
// over the four nodes around the txz point; Cerjan taper from the layer
// tables.  The step is two passes (velocity, then stress with the new
// velocities), one point per thread with read-only-cache loads: 2D grids are
// small enough that the L1/L2 hold every reused row.  dt_sign = -1 runs the
// transposed step in the (b_avg vbar, g C tbar) variables (the taper, C and
// the averages are pointwise), which adjoint modelling uses.
#include "common.cuh"

namespace {

constexpr int BZ = 32, BXR = 8;       // block: 32 z x 8 x

WP_DEV float at2(const float *__restrict__ f, const GridDev &g, int x, int z)
{
    return (x >= 0 && x < g.NX && z >= 0 && z < g.NZ) ? __ldg(f + (long long)x * g.NZ + z) : 0.f;
}

// v <- g (v + c b_avg Dtau(tau)),  c = dt / h (signed)
template <int M>
__global__ void __launch_bounds__(BZ * BXR)
el2_vpass(GridDev g, FDW w, float *vx, float *vz, const float *__restrict__ txx, const float *__restrict__ tzz,
          const float *__restrict__ txz, const float *__restrict__ bu, float c)
{
    const int z = blockIdx.x * BZ + threadIdx.x, x = blockIdx.y * BXR + threadIdx.y;
    if (z >= g.NZ || x >= g.NX) return;
    const long long q = (long long)x * g.NZ + z;
    float dx = 0.f, dz = 0.f;
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const float b = w.b[k - 1];
        // vx: D+x txx + D-z txz ;  vz: D-x txz + D+z tzz
        dx += b * ((at2(txx, g, x + k, z) - at2(txx, g, x - k + 1, z)) +
                   (at2(txz, g, x, z + k - 1) - at2(txz, g, x, z - k)));
        dz += b * ((at2(txz, g, x + k - 1, z) - at2(txz, g, x - k, z)) +
                   (at2(tzz, g, x, z + k) - at2(tzz, g, x, z - k + 1)));
    }
    const float b0 = __ldg(bu + q);
    const float bx = 0.5f * (b0 + __ldg(bu + (long long)min(x + 1, g.NX - 1) * g.NZ + z));
    const float bz = 0.5f * (b0 + __ldg(bu + (long long)x * g.NZ + min(z + 1, g.NZ - 1)));
    const float *tz = g.tab + 2 * (g.NX + g.NY);
    const float gy = __ldg(g.tab + 2 * g.NX);
    const float gvx = __ldg(g.tab + 2 * x + 1) * gy * __ldg(tz + 2 * z);
    const float gvz = __ldg(g.tab + 2 * x) * gy * __ldg(tz + 2 * z + 1);
    vx[q] = gvx * (vx[q] + c * bx * dx);
    vz[q] = gvz * (vz[q] + c * bz * dz);
}

// tau <- g (tau + c C S(v)),  c = dt / h (signed)
template <int M>
__global__ void __launch_bounds__(BZ * BXR)
el2_tpass(GridDev g, FDW w, const float *__restrict__ vx, const float *__restrict__ vz, float *txx, float *tzz,
          float *txz, const float *__restrict__ lam, const float *__restrict__ mu, float c, int *flag, int check)
{
    const int z = blockIdx.x * BZ + threadIdx.x, x = blockIdx.y * BXR + threadIdx.y;
    if (z >= g.NZ || x >= g.NX) return;
    const long long q = (long long)x * g.NZ + z;
    float exx = 0.f, ezz = 0.f, gxz = 0.f;
#pragma unroll
    for (int k = 1; k <= M; k++) {
        const float b = w.b[k - 1];
        exx += b * (at2(vx, g, x + k - 1, z) - at2(vx, g, x - k, z));
        ezz += b * (at2(vz, g, x, z + k - 1) - at2(vz, g, x, z - k));
        gxz += b * ((at2(vx, g, x, z + k) - at2(vx, g, x, z - k + 1)) +
                    (at2(vz, g, x + k, z) - at2(vz, g, x - k + 1, z)));
    }
    const int x1 = min(x + 1, g.NX - 1), z1 = min(z + 1, g.NZ - 1);
    const float mxz = 0.25f * ((__ldg(mu + q) + __ldg(mu + (long long)x * g.NZ + z1)) +
                               (__ldg(mu + (long long)x1 * g.NZ + z) + __ldg(mu + (long long)x1 * g.NZ + z1)));
    const float l = __ldg(lam + q), m = __ldg(mu + q), tr = exx + ezz;
    const float *tz = g.tab + 2 * (g.NX + g.NY);
    const float gy = __ldg(g.tab + 2 * g.NX);
    const float gn = __ldg(g.tab + 2 * x) * gy * __ldg(tz + 2 * z);
    const float gxzt = __ldg(g.tab + 2 * x + 1) * gy * __ldg(tz + 2 * z + 1);
    const float a = gn * (txx[q] + c * (l * tr + 2.f * m * exx));
    const float d = gn * (tzz[q] + c * (l * tr + 2.f * m * ezz));
    const float e = gxzt * (txz[q] + c * mxz * gxz);
    txx[q] = a;
    tzz[q] = d;
    txz[q] = e;
    if (check && !(isfinite(a) && isfinite(d) && isfinite(e))) atomicOr(flag, 1);
}

template <int M>
int launch(prop_s *P, float *const *S, float dt_sign)
{
    const GridDev &g = P->g;
    dim3 blk(BZ, BXR), grd((g.NZ + BZ - 1) / BZ, (g.NX + BXR - 1) / BXR);
    const float c = dt_sign * g.dt * g.ih;
    el2_vpass<M><<<grd, blk, 0, P->stream>>>(g, P->w, S[0], S[1], S[2], S[3], S[4], P->bu, c);
    el2_tpass<M><<<grd, blk, 0, P->stream>>>(g, P->w, S[0], S[1], S[2], S[3], S[4], P->lam, P->mu, c, P->flag,
                                             P->d.check_nan);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// one 2D elastic step of S = (vx, vz, txx, tzz, txz) in place; dt_sign = -1:
// the transposed step in the adjoint-modelling variables
int el2_launch(prop_s *P, float *const *S, float dt_sign)
{
    prof_begin(P, dt_sign > 0 ? 2 : 5);
    int rc;
    switch (P->M) {
    case 2: rc = launch<2>(P, S, dt_sign); break;
    case 4: rc = launch<4>(P, S, dt_sign); break;
    case 6: rc = launch<6>(P, S, dt_sign); break;
    case 8: rc = launch<8>(P, S, dt_sign); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, dt_sign > 0 ? 2 : 5);
    return rc;
}
