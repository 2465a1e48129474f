// Elastic step passes with software pipelining (Sec. IV, Eq. elas1).
//
// Two passes per step, each streaming along x over a 32(z) x 16(y) tile:
//   velocity pass  v <- g (v + dt b_avg Dtau(tau))
//   stress pass    tau <- g (tau + dt C S(v))
// The transposed step (adjoint modelling) is the same two passes with
// dt -> -dt in the variables (b_avg vbar, g C tbar).  These kernels serve
// grids whose computational NZ is not a multiple of 4 (the TMA-fed passes
// need 16-byte rows).
//
// Pipelining: while plane x is computed from shared memory, the loads of
// plane x+1 (x-queue heads, own interior values, an even share of the halo
// elements, pointwise fields) are already in flight in registers; shared
// planes are double-buffered so one barrier per plane suffices.  Buoyancy
// and mu enter through small shared planes with a +1 row/column so that the
// face and edge averages need no extra global loads.
#include "common.cuh"

namespace {

constexpr int FZ = 32, FY = 16, NT = FZ * FY;

WP_DEV bool inside(const GridDev &g, int x, int y, int z)
{
    return x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ;
}
WP_DEV float lz(const float *__restrict__ f, const GridDev &g, int x, int y, int z)
{
    return inside(g, x, y, z) ? __ldg(f + gidx(g, x, y, z)) : 0.f;
}
// clamped load (parameters are extended by edge replication)
WP_DEV float lc(const float *__restrict__ f, const GridDev &g, int x, int y, int z)
{
    x = min(max(x, 0), g.NX - 1);
    y = min(max(y, 0), g.NY - 1);
    z = min(max(z, 0), g.NZ - 1);
    return __ldg(f + gidx(g, x, y, z));
}
WP_DEV float tp(const GridDev &g, int x, int hx, int y, int hy, int z, int hz)
{
    return __ldg(g.tab + 2 * x + hx) * __ldg(g.tab + 2 * g.NX + 2 * y + hy) *
           __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * z + hz);
}

struct F9 {
    float *f[9];
};

// Shared-plane geometry.  kind 0: y halo (rows FY+2M, cols FZ); kind 1: z
// halo (rows FY, cols FZ+2M); kind 2: cross (rows FY+2M, cols FZ+2M);
// kind 3: +1 plane (rows FY+1, cols FZ+1; interior plus the row y0+FY and
// the column z0+FZ).
template <int M>
struct PG {
    static constexpr int rows(int k) { return k == 1 ? FY : (k == 3 ? FY + 1 : FY + 2 * M); }
    static constexpr int cols(int k) { return k == 0 ? FZ : (k == 3 ? FZ + 1 : FZ + 2 * M); }
    static constexpr int size(int k) { return rows(k) * cols(k); }
    static constexpr int nhalo(int k)
    {
        return k == 3 ? FZ + FY + 1 : (k != 1 ? 2 * M * FZ : 0) + (k != 0 ? 2 * M * FY : 0);
    }
    // interior offset of thread (ty, tz)
    static WP_DEV int inner(int k, int ty, int tz)
    {
        const int r = (k == 0 || k == 2) ? ty + M : ty;
        const int c = (k == 1 || k == 2) ? tz + M : tz;
        return r * cols(k) + c;
    }
};

// decode halo element i of field k into (smem offset within the field, dy, dz)
template <int M>
WP_DEV void halo_at(int k, int i, int &off, int &dy, int &dz)
{
    const int cols = PG<M>::cols(k);
    if (k == 3) {
        if (i <= FZ) { off = FY * cols + i; dy = FY; dz = i; }      // row y0+FY incl. corner
        else { i -= FZ + 1; off = i * cols + FZ; dy = i; dz = FZ; }
        return;
    }
    if (k != 1) {
        const int n = 2 * M * FZ;
        if (i < n) {
            const int r = i / FZ, c = i % FZ;
            const int row = r < M ? r : r + FY;
            dy = r < M ? r - M : FY + r - M;
            dz = c;
            off = row * cols + (k == 2 ? c + M : c);
            return;
        }
        i -= n;
    }
    const int r = i / (2 * M), cc = i % (2 * M);
    const int col = cc < M ? cc : cc + FZ;
    dy = r;
    dz = cc < M ? cc - M : FZ + cc - M;
    off = (k == 2 ? r + M : r) * cols + col;
}

// Per-thread share of the halo elements of NF fields with kinds K[].
// (fld + 1) << 20 | (dy + 64) << 10 | (dz + 64) packed in one int; off in another
template <int M, int NF, int S>
struct HaloShare {
    int code[S], off[S];
    WP_DEV int fld(int s) const { return (code[s] >> 20) - 1; }
    WP_DEV int dy(int s) const { return ((code[s] >> 10) & 1023) - 64; }
    WP_DEV int dz(int s) const { return (code[s] & 1023) - 64; }
    template <class KF, class BF>
    WP_DEV void init(KF K, BF base, int tid)
    {
        int total = 0;
        for (int k = 0; k < NF; k++) total += PG<M>::nhalo(K(k));
#pragma unroll
        for (int s = 0; s < S; s++) {
            int i = tid + s * NT;
            code[s] = 0;
            off[s] = 0;
            if (i >= total) continue;
            for (int k = 0; k < NF; k++) {
                const int n = PG<M>::nhalo(K(k));
                if (i < n) {
                    int o, dy_, dz_;
                    halo_at<M>(K(k), i, o, dy_, dz_);
                    code[s] = ((k + 1) << 20) | ((dy_ + 64) << 10) | (dz_ + 64);
                    off[s] = base(k) + o;
                    break;
                }
                i -= n;
            }
        }
    }
};

// ---------------------------------------------------------------------------
// velocity pass
// fields: 0 f_xy (y halo), 1 f_yy (y), 2 f_yz (cross), 3 f_xz (z), 4 f_zz (z),
//         5 buoyancy (+1 plane)
// ---------------------------------------------------------------------------
template <int M>
struct VP {
    static constexpr int NF = 6;
    static constexpr int B0 = 0, B1 = PG<M>::size(0), B2 = 2 * PG<M>::size(0),
                         B3 = B2 + PG<M>::size(2), B4 = B3 + PG<M>::size(1),
                         B5 = B4 + PG<M>::size(1), BUF = B5 + PG<M>::size(3);
    static constexpr int HTOT = 2 * PG<M>::nhalo(0) + PG<M>::nhalo(2) + 2 * PG<M>::nhalo(1) +
                                PG<M>::nhalo(3);
    static constexpr int S = (HTOT + NT - 1) / NT;
};

// stress component c at (x, y, z), 0 outside the grid.
// Components: 0 xx 1 yy 2 zz 3 xy 4 xz 5 yz
WP_DEV const float *pick(const F9 &s, int i)
{
    switch (i) {
    case 0: return s.f[0]; case 1: return s.f[1]; case 2: return s.f[2];
    case 3: return s.f[3]; case 4: return s.f[4]; case 5: return s.f[5];
    case 6: return s.f[6]; case 7: return s.f[7];
    }
    return s.f[8];
}

WP_DEV float vp_val(const GridDev &g, const F9 &s, int c, int x, int y, int z)
{
    return inside(g, x, y, z) ? __ldg(pick(s, 3 + c) + gidx(g, x, y, z)) : 0.f;
}

template <int M>
__global__ void __launch_bounds__(NT, 2)
el_vpass(GridDev g, FDW w, F9 s, const float *__restrict__ bu, int xc)
{
    using L = VP<M>;
    constexpr int Q = 2 * M, NF = L::NF, S = L::S;
    extern __shared__ float sm[];
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    // field -> stress component (for vp_val); field 5 = buoyancy
    auto comp = [](int f) { return f == 0 ? 3 : f == 1 ? 1 : f == 2 ? 5 : f == 3 ? 4 : 2; };
    HaloShare<M, NF, S> hs;
    hs.init([](int k) { return k < 2 ? 0 : k == 2 ? 2 : k < 5 ? 1 : 3; },
            [](int k) {
                return k == 0 ? L::B0 : k == 1 ? L::B1 : k == 2 ? L::B2 : k == 3 ? L::B3
                       : k == 4 ? L::B4 : L::B5;
            },
            tid);

    float qxx[Q], qxy[Q], qxz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qxx[j] = vp_val(g, s, 0, xa - M + 1 + j, y, z);
        qxy[j] = vp_val(g, s, 3, xa - M + j, y, z);
        qxz[j] = vp_val(g, s, 4, xa - M + j, y, z);
    }
    // prefetched values of the next plane
    float nxx, nxy, nxz, nyy, nzz, nyz, nb = 0.f, nbx = 0.f, hv[S];
    auto fetch = [&](int x) {
        nxx = vp_val(g, s, 0, x + M, y, z);
        nxy = vp_val(g, s, 3, x + M - 1, y, z);
        nxz = vp_val(g, s, 4, x + M - 1, y, z);
        nyy = vp_val(g, s, 1, x, y, z);
        nzz = vp_val(g, s, 2, x, y, z);
        nyz = vp_val(g, s, 5, x, y, z);
        nb = lc(bu, g, x, y, z);
        nbx = lc(bu, g, x + 1, y, z);
#pragma unroll
        for (int k = 0; k < S; k++) {
            const int f = hs.fld(k);
            float v = 0.f;
            if (f >= 0) {
                const int yy = y0 + hs.dy(k), zz = z0 + hs.dz(k);
                v = f == 5 ? lc(bu, g, x, yy, zz) : vp_val(g, s, comp(f), x, yy, zz);
            }
            hv[k] = v;
        }
    };
    fetch(xa);
    const bool act = y < g.NY && z < g.NZ;
    const float c = g.dt * g.ih;
    for (int x = xa; x < xb; x++) {
        float *B = sm + ((x - xa) & 1) * L::BUF;
        qxx[Q - 1] = nxx;
        qxy[Q - 1] = nxy;
        qxz[Q - 1] = nxz;
        B[L::B0 + PG<M>::inner(0, ty, tz)] = qxy[M];
        B[L::B1 + PG<M>::inner(0, ty, tz)] = nyy;
        B[L::B2 + PG<M>::inner(2, ty, tz)] = nyz;
        B[L::B3 + PG<M>::inner(1, ty, tz)] = qxz[M];
        B[L::B4 + PG<M>::inner(1, ty, tz)] = nzz;
        B[L::B5 + PG<M>::inner(3, ty, tz)] = nb;
#pragma unroll
        for (int k = 0; k < S; k++)
            if (hs.fld(k) >= 0) B[hs.off[k]] = hv[k];
        const float bxn = nbx;
        __syncthreads();
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
        const long long qv = act ? gidx(g, x, y, z) : 0;
        if (act) {
            v0 = s.f[0][qv];
            v1 = s.f[1][qv];
            v2 = s.f[2][qv];
        }
        if (x + 1 < xb) fetch(x + 1);
        if (act) {
            const float *sxy = B + L::B0, *syy = B + L::B1, *syz = B + L::B2, *sxz = B + L::B3,
                        *szz = B + L::B4;
            constexpr int C0 = PG<M>::cols(0), C1 = PG<M>::cols(1), C2 = PG<M>::cols(2);
            const int cy = ty + M, cz = tz + M;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float b = w.b[k - 1];
                d0 += b * ((qxx[M - 1 + k] - qxx[M - k]) +
                           (sxy[(cy + k - 1) * C0 + tz] - sxy[(cy - k) * C0 + tz]) +
                           (sxz[ty * C1 + cz + k - 1] - sxz[ty * C1 + cz - k]));
                d1 += b * ((qxy[M + k - 1] - qxy[M - k]) +
                           (syy[(cy + k) * C0 + tz] - syy[(cy - k + 1) * C0 + tz]) +
                           (syz[cy * C2 + cz + k - 1] - syz[cy * C2 + cz - k]));
                d2 += b * ((qxz[M + k - 1] - qxz[M - k]) +
                           (syz[(cy + k - 1) * C2 + cz] - syz[(cy - k) * C2 + cz]) +
                           (szz[ty * C1 + cz + k] - szz[ty * C1 + cz - k + 1]));
            }
            const long long q = gidx(g, x, y, z);
            constexpr int C3 = PG<M>::cols(3);
            const float *sb = B + L::B5;
            const float b0 = sb[ty * C3 + tz];
            const float bx = 0.5f * (b0 + bxn);
            const float by = 0.5f * (b0 + sb[(y + 1 < g.NY ? ty + 1 : ty) * C3 + tz]);
            const float bz = 0.5f * (b0 + sb[ty * C3 + (z + 1 < g.NZ ? tz + 1 : tz)]);
            s.f[0][q] = tp(g, x, 1, y, 0, z, 0) * (v0 + c * bx * d0);
            s.f[1][q] = tp(g, x, 0, y, 1, z, 0) * (v1 + c * by * d1);
            s.f[2][q] = tp(g, x, 0, y, 0, z, 1) * (v2 + c * bz * d2);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qxx[j] = qxx[j + 1];
            qxy[j] = qxy[j + 1];
            qxz[j] = qxz[j + 1];
        }
    }
}

// ---------------------------------------------------------------------------
// stress pass
// fields: 0 f_vx, 1 f_vy, 2 f_vz (cross); 3 mu plane (+1) -- ring of 3
// ---------------------------------------------------------------------------
template <int M>
struct TP_ {
    static constexpr int B0 = 0, B1 = PG<M>::size(2), B2 = 2 * PG<M>::size(2),
                         BUF = 3 * PG<M>::size(2);
    static constexpr int MU = PG<M>::size(3);   // one mu plane
    static constexpr int HTOT = 3 * PG<M>::nhalo(2);
    static constexpr int S = (HTOT + NT - 1) / NT;
    static constexpr int SMU = (PG<M>::nhalo(3) + NT - 1) / NT;
};

// velocity component c at (x, y, z), 0 outside the grid
WP_DEV float tp_val(const GridDev &g, const F9 &s, int c, int x, int y, int z)
{
    return inside(g, x, y, z) ? __ldg(pick(s, c) + gidx(g, x, y, z)) : 0.f;
}

template <int M>
__global__ void __launch_bounds__(NT, 2)
el_tpass(GridDev g, FDW w, F9 s, const float *__restrict__ lam, const float *__restrict__ mu, int xc)
{
    using L = TP_<M>;
    constexpr int Q = 2 * M, S = L::S;
    constexpr int C2 = PG<M>::cols(2), C3 = PG<M>::cols(3);
    extern __shared__ float sm[];
    float *smu = sm + 2 * L::BUF;            // ring of 3 mu planes
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    HaloShare<M, 3, S> hs;
    hs.init([](int) { return 2; }, [](int k) { return k * PG<M>::size(2); }, tid);
    // +1 share of the mu plane: element tid < FZ + FY
    int muo = -1, mudy = 0, mudz = 0;
    if (tid < PG<M>::nhalo(3)) halo_at<M>(3, tid, muo, mudy, mudz);

    float qvx[Q], qvy[Q], qvz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        qvx[j] = tp_val(g, s, 0, xa - M + j, y, z);
        qvy[j] = tp_val(g, s, 1, xa - M + 1 + j, y, z);
        qvz[j] = tp_val(g, s, 2, xa - M + 1 + j, y, z);
    }
    float nvx, nvy, nvz, hv[S], nmu, nmuh;
    auto fetch = [&](int x) {
        nvx = tp_val(g, s, 0, x + M - 1, y, z);
        nvy = tp_val(g, s, 1, x + M, y, z);
        nvz = tp_val(g, s, 2, x + M, y, z);
#pragma unroll
        for (int k = 0; k < S; k++) {
            const int f = hs.fld(k);
            hv[k] = f >= 0 ? tp_val(g, s, f, x, y0 + hs.dy(k), z0 + hs.dz(k)) : 0.f;
        }
        // mu plane x+1 (clamped) for the edge averages
        nmu = lc(mu, g, x + 1, y, z);
        nmuh = muo >= 0 ? lc(mu, g, x + 1, y0 + mudy, z0 + mudz) : 0.f;
    };
    // mu plane xa into ring slot xa % 3
    {
        float *R = smu + (xa % 3) * L::MU;
        R[PG<M>::inner(3, ty, tz)] = lc(mu, g, xa, y, z);
        if (muo >= 0) R[muo] = lc(mu, g, xa, y0 + mudy, z0 + mudz);
    }
    fetch(xa);
    const bool act = y < g.NY && z < g.NZ;
    const float c = g.dt * g.ih;
    const int y1 = y + 1 < g.NY ? ty + 1 : ty, z1 = z + 1 < g.NZ ? tz + 1 : tz;
    for (int x = xa; x < xb; x++) {
        float *B = sm + ((x - xa) & 1) * L::BUF;
        qvx[Q - 1] = nvx;
        qvy[Q - 1] = nvy;
        qvz[Q - 1] = nvz;
        B[L::B0 + PG<M>::inner(2, ty, tz)] = qvx[M];
        B[L::B1 + PG<M>::inner(2, ty, tz)] = qvy[M - 1];
        B[L::B2 + PG<M>::inner(2, ty, tz)] = qvz[M - 1];
#pragma unroll
        for (int k = 0; k < S; k++)
            if (hs.fld(k) >= 0) B[hs.off[k]] = hv[k];
        {
            float *R = smu + ((x + 1) % 3) * L::MU;
            R[PG<M>::inner(3, ty, tz)] = nmu;
            if (muo >= 0) R[muo] = nmuh;
        }
        __syncthreads();
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, t4 = 0.f, t5 = 0.f, l = 0.f;
        const long long qt = act ? gidx(g, x, y, z) : 0;
        if (act) {
            t0 = s.f[3][qt]; t1 = s.f[4][qt]; t2 = s.f[5][qt];
            t3 = s.f[6][qt]; t4 = s.f[7][qt]; t5 = s.f[8][qt];
            l = __ldg(lam + qt);
        }
        if (x + 1 < xb) fetch(x + 1);
        if (act) {
            const float *svx = B + L::B0, *svy = B + L::B1, *svz = B + L::B2;
            const int cy = ty + M, cz = tz + M;
            float exx = 0.f, eyy = 0.f, ezz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float b = w.b[k - 1];
                exx += b * (qvx[M + k - 1] - qvx[M - k]);
                eyy += b * (svy[(cy + k - 1) * C2 + cz] - svy[(cy - k) * C2 + cz]);
                ezz += b * (svz[cy * C2 + cz + k - 1] - svz[cy * C2 + cz - k]);
                gxy += b * ((svx[(cy + k) * C2 + cz] - svx[(cy - k + 1) * C2 + cz]) +
                            (qvy[M - 1 + k] - qvy[M - k]));
                gxz += b * ((svx[cy * C2 + cz + k] - svx[cy * C2 + cz - k + 1]) +
                            (qvz[M - 1 + k] - qvz[M - k]));
                gyz += b * ((svy[cy * C2 + cz + k] - svy[cy * C2 + cz - k + 1]) +
                            (svz[(cy + k) * C2 + cz] - svz[(cy - k + 1) * C2 + cz]));
            }
            const float *R0 = smu + (x % 3) * L::MU;
            const float *R1 = smu + ((x + 1 < g.NX ? x + 1 : x) % 3) * L::MU;
            const float m0 = R0[ty * C3 + tz], my = R0[y1 * C3 + tz], mz = R0[ty * C3 + z1];
            const float mx = R1[ty * C3 + tz], mxy_ = R1[y1 * C3 + tz], mxz_ = R1[ty * C3 + z1];
            const float myz_ = R0[y1 * C3 + z1];
            const float mxy = 0.25f * (m0 + mx + my + mxy_);
            const float mxz = 0.25f * (m0 + mx + mz + mxz_);
            const float myz = 0.25f * (m0 + my + mz + myz_);
            const float tr = exx + eyy + ezz, m2 = 2.f * m0;
            const long long q = gidx(g, x, y, z);
            const float gn = tp(g, x, 0, y, 0, z, 0);
            const float gxy_ = tp(g, x, 1, y, 1, z, 0), gxz_ = tp(g, x, 1, y, 0, z, 1),
                        gyz_ = tp(g, x, 0, y, 1, z, 1);
            s.f[3][q] = gn * (t0 + c * (l * tr + m2 * exx));
            s.f[4][q] = gn * (t1 + c * (l * tr + m2 * eyy));
            s.f[5][q] = gn * (t2 + c * (l * tr + m2 * ezz));
            s.f[6][q] = gxy_ * (t3 + c * mxy * gxy);
            s.f[7][q] = gxz_ * (t4 + c * mxz * gxz);
            s.f[8][q] = gyz_ * (t5 + c * myz * gyz);
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
int launch(prop_s *P, float *const *S, float dt_sign)
{
    GridDev g = P->g;
    g.dt = dt_sign * g.dt;
    const int xc = P->xchunk;
    dim3 blk(FZ, FY, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    F9 s;
    for (int i = 0; i < 9; i++) s.f[i] = S[i];
    const size_t smv = 2 * VP<M>::BUF * sizeof(float);
    const size_t smt = (2 * TP_<M>::BUF + 3 * TP_<M>::MU) * sizeof(float);
    static const bool attr = (cudaFuncSetAttribute(el_vpass<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv),
                              cudaFuncSetAttribute(el_tpass<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt), true);
    (void)attr;
    prof_begin(P, dt_sign > 0 ? 2 : 5);
    el_vpass<M><<<grd, blk, smv, P->stream>>>(g, P->w, s, P->bu, xc);
    el_tpass<M><<<grd, blk, smt, P->stream>>>(g, P->w, s, P->lam, P->mu, xc);
    prof_end(P, dt_sign > 0 ? 2 : 5);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// elastic step with time step dt_sign * dt, in place on S (9 fields):
// forward (+1), or the transposed step in (b_avg vbar, g C tbar) (-1)
int el_launch_fast(prop_s *P, float *const *S, float dt_sign)
{
    switch (P->M) {
    case 2: return launch<2>(P, S, dt_sign);
    case 4: return launch<4>(P, S, dt_sign);
    case 6: return launch<6>(P, S, dt_sign);
    case 8: return launch<8>(P, S, dt_sign);
    }
    return wp_fail(P, PROP_EINVAL, "unsupported space order");
}
