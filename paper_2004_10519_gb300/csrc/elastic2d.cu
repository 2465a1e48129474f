// 2D elastic propagator (x-z plane): the velocity-stress system of Sec. IV-A
// (Eq. elas1, elastic listing) with every y term dropped, as in the 2D
// example of Sec. IV-B.  Fields on the staggered grid of the 3D system:
// vx at (x+1/2, z), vz at (x, z+1/2), txx and tzz at nodes, txz at
// (x+1/2, z+1/2); b averaged over the two nodes of a velocity point, mu
// over the four nodes around the txz point; Cerjan taper from the layer
// tables.  The step is two passes (velocity, then stress with the new
// velocities) over 32 x 32 tiles staged in shared memory with their halos
// (2D working sets mostly sit in L2).  dt_sign = -1 runs the
// transposed step in the (b_avg vbar, g C tbar) variables (the taper, C and
// the averages are pointwise), which adjoint modelling uses.
#include "common.cuh"

namespace {

// Tile of 32 (z) x 32 (x) points per CTA of 32 x 8 threads (four x points
// per thread).  Each differentiated field is staged once in shared memory
// with its halo (zero outside the grid = the zero extension of the
// operators); the taps then read shared rows (one wavefront per warp
// access) instead of unaligned read-only-cache loads.
constexpr int TZ = 32, TXR = 32, BXR = 8;

template <int M>
struct Tile2 {
    static constexpr int R = TXR + 2 * M, C = TZ + 2 * M;   // rows (x), columns (z) with halo
};

// stage f[x0 - HX .. x0 + TXR + HX) x [z0 - HZ .. z0 + TZ + HZ) into s (row
// pitch TZ + 2 HZ); a fixed trip count lets every load of a thread be in
// flight before its shared stores
template <int HX, int HZ>
WP_DEV void stage(float *s, const float *__restrict__ f, const GridDev &g, int x0, int z0)
{
    constexpr int cols = TZ + 2 * HZ, n = (TXR + 2 * HX) * cols, NTH = TZ * BXR, IT = (n + NTH - 1) / NTH;
    const int tid = threadIdx.y * TZ + threadIdx.x;
    float v[IT];
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int i = tid + it * NTH, r = i / cols, c = i % cols;
        const int x = x0 - HX + r, z = z0 - HZ + c;
        v[it] = (i < n && x >= 0 && x < g.NX && z >= 0 && z < g.NZ) ? __ldg(f + (long long)x * g.NZ + z) : 0.f;
    }
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int i = tid + it * NTH;
        if (i < n) s[i] = v[it];
    }
}

// v <- g (v + c b_avg Dtau(tau)),  c = dt / h (signed)
template <int M>
__global__ void __launch_bounds__(TZ * BXR)
el2_vpass(GridDev g, FDW w, float *vx, float *vz, const float *__restrict__ txx, const float *__restrict__ tzz,
          const float *__restrict__ txz, const float *__restrict__ bu, float c)
{
    using T = Tile2<M>;
    __shared__ float sxx[T::R * TZ], sxz[T::R * T::C], szz[TXR * T::C];
    const int z0 = blockIdx.x * TZ, x0 = blockIdx.y * TXR;
    stage<M, 0>(sxx, txx, g, x0, z0);
    stage<M, M>(sxz, txz, g, x0, z0);
    stage<0, M>(szz, tzz, g, x0, z0);
    __syncthreads();
    const int tz = threadIdx.x, z = z0 + tz;
    if (z >= g.NZ) return;
    const float *tzt = g.tab + 2 * (g.NX + g.NY);
    const float gy = __ldg(g.tab + 2 * g.NX), gzn = __ldg(tzt + 2 * z), gzh = __ldg(tzt + 2 * z + 1);
    const int z1 = min(z + 1, g.NZ - 1);
#pragma unroll
    for (int j = 0; j < TXR / BXR; j++) {
        const int r = threadIdx.y * (TXR / BXR) + j, x = x0 + r;
        if (x >= g.NX) break;
        float dx = 0.f, dz = 0.f;
        const float *rxx = sxx + (r + M) * TZ + tz, *rxz = sxz + (r + M) * T::C + tz + M,
                    *rzz = szz + r * T::C + tz + M;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const float b = w.b[k - 1];
            // vx: D+x txx + D-z txz ;  vz: D-x txz + D+z tzz
            dx += b * ((rxx[k * TZ] - rxx[(1 - k) * TZ]) + (rxz[k - 1] - rxz[-k]));
            dz += b * ((rxz[(k - 1) * T::C] - rxz[-k * T::C]) + (rzz[k] - rzz[1 - k]));
        }
        const long long q = (long long)x * g.NZ + z;
        const float b0 = __ldg(bu + q);
        const float bx = 0.5f * (b0 + __ldg(bu + (long long)min(x + 1, g.NX - 1) * g.NZ + z));
        const float bz = 0.5f * (b0 + __ldg(bu + (long long)x * g.NZ + z1));
        const float gvx = __ldg(g.tab + 2 * x + 1) * gy * gzn;
        const float gvz = __ldg(g.tab + 2 * x) * gy * gzh;
        vx[q] = gvx * (vx[q] + c * bx * dx);
        vz[q] = gvz * (vz[q] + c * bz * dz);
    }
}

// tau <- g (tau + c C S(v)),  c = dt / h (signed)
template <int M>
__global__ void __launch_bounds__(TZ * BXR)
el2_tpass(GridDev g, FDW w, const float *__restrict__ vx, const float *__restrict__ vz, float *txx, float *tzz,
          float *txz, const float *__restrict__ lam, const float *__restrict__ mu, float c, int *flag, int check)
{
    using T = Tile2<M>;
    __shared__ float svx[T::R * T::C], svz[T::R * T::C];
    const int z0 = blockIdx.x * TZ, x0 = blockIdx.y * TXR;
    stage<M, M>(svx, vx, g, x0, z0);
    stage<M, M>(svz, vz, g, x0, z0);
    __syncthreads();
    const int tz = threadIdx.x, z = z0 + tz;
    if (z >= g.NZ) return;
    const float *tzt = g.tab + 2 * (g.NX + g.NY);
    const float gy = __ldg(g.tab + 2 * g.NX), gzn = __ldg(tzt + 2 * z), gzh = __ldg(tzt + 2 * z + 1);
    const int z1 = min(z + 1, g.NZ - 1);
#pragma unroll
    for (int j = 0; j < TXR / BXR; j++) {
        const int r = threadIdx.y * (TXR / BXR) + j, x = x0 + r;
        if (x >= g.NX) break;
        const float *rvx = svx + (r + M) * T::C + tz + M, *rvz = svz + (r + M) * T::C + tz + M;
        float exx = 0.f, ezz = 0.f, gxz = 0.f;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const float b = w.b[k - 1];
            exx += b * (rvx[(k - 1) * T::C] - rvx[-k * T::C]);
            ezz += b * (rvz[k - 1] - rvz[-k]);
            gxz += b * ((rvx[k] - rvx[1 - k]) + (rvz[k * T::C] - rvz[(1 - k) * T::C]));
        }
        const long long q = (long long)x * g.NZ + z;
        const int x1 = min(x + 1, g.NX - 1);
        const float mxz = 0.25f * ((__ldg(mu + q) + __ldg(mu + (long long)x * g.NZ + z1)) +
                                   (__ldg(mu + (long long)x1 * g.NZ + z) + __ldg(mu + (long long)x1 * g.NZ + z1)));
        const float l = __ldg(lam + q), m = __ldg(mu + q), tr = exx + ezz;
        const float gn = __ldg(g.tab + 2 * x) * gy * gzn;
        const float gxzt = __ldg(g.tab + 2 * x + 1) * gy * gzh;
        const float a = gn * (txx[q] + c * (l * tr + 2.f * m * exx));
        const float d = gn * (tzz[q] + c * (l * tr + 2.f * m * ezz));
        const float e = gxzt * (txz[q] + c * mxz * gxz);
        txx[q] = a;
        tzz[q] = d;
        txz[q] = e;
        if (check && !(isfinite(a) && isfinite(d) && isfinite(e))) atomicOr(flag, 1);
    }
}

template <int M>
int launch(prop_s *P, float *const *S, float dt_sign)
{
    const GridDev &g = P->g;
    dim3 blk(TZ, BXR), grd((g.NZ + TZ - 1) / TZ, (g.NX + TXR - 1) / TXR);
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
