// Stencil passes fed by the Tensor Memory Accelerator (sm_103a).
//
// Each CTA owns a 32(z) x 16(y) tile of columns and streams along x.  For
// every plane the y/z-halo boxes of the differentiated fields are fetched by
// one thread with cp.async.bulk.tensor into a 3-stage shared-memory ring
// (mbarrier completion); out-of-grid elements arrive as zeros, which is the
// zero extension of the finite-difference operators.  Threads only do
// arithmetic on shared memory; x-derivatives use per-thread register queues
// fed by plain coalesced loads, pointwise fields are plain loads issued one
// plane ahead.  Every mbarrier wait is bounded in time: on expiry the CTA
// sets bit 2 of the error word and leaves (no hang).
//
// Elastic (Sec. IV, Eq. elas1, elastic listing):
//   velocity pass  v <- g (v + dt b_avg Dtau(tau))
//   stress pass    tau <- g (tau + dt C S(v))
// The transposed step is the same two passes with dt -> -dt in the variables
// (b_avg vbar, g C tbar) (the taper, C and the averages are pointwise and
// commute), so adjoint modelling uses these kernels too.
// TTI (Sec. III-A): rotation pass (D of p, r or of zeta = C lam) and update
// pass (divergence, coupling, damped leapfrog, fused imaging).
#include "tile.cuh"

#include <cuda.h>
#include <cstdlib>
#include <mutex>

namespace {

using namespace tile;

constexpr int NSTAGE = 3;

struct F9 {
    float *f[9];
};

// ---------------------------------------------------------------------------
// device: mbarrier / TMA helpers (inline PTX)
// ---------------------------------------------------------------------------
WP_DEV uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

WP_DEV void mbar_init(uint64_t *bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
WP_DEV void fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
WP_DEV void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}
WP_DEV void tma3(float *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            saddr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
        : "memory");
}
WP_DEV bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
WP_DEV uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of bar; false after ~2 s
WP_DEV bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > 2000000000ull) return false;
    return true;
}

constexpr int al32(int n) { return (n + 31) & ~31; }   // 128-byte aligned float offsets

// box geometries (floats): rows x cols
template <int M>
struct BX {
    static constexpr int MZ = (M + 3) & ~3;                     // z halo rounded to 16 bytes
    static constexpr int YR = FY + 2 * M, YC = FZ;              // y-halo box
    static constexpr int ZR = FY, ZC = FZ + 2 * MZ;             // z-halo box
    static constexpr int RR = FY + 2 * M, RC = FZ + 2 * MZ;     // rectangle (y and z halo)
    static constexpr int PR = FY + 1, PC = FZ + 4;              // +1 box (interior + row/col)
    static constexpr int YS = al32(YR * YC), ZS = al32(ZR * ZC), RS = al32(RR * RC), PS = al32(PR * PC);
};

// one bounded wait of the whole CTA for stage `st` of iteration `it`;
// returns false (uniformly) if any thread gave up
WP_DEV bool stage_wait(uint64_t *bars, int it, int *err)
{
    const int st = it % NSTAGE;
    const bool ok = mbar_wait(&bars[st], (uint32_t)((it / NSTAGE) & 1));
    const int bad = __syncthreads_or(!ok);
    if (bad) {
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(err, 2);
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// elastic velocity pass
// stage: [xy (y box)] [yy (y box)] [xz (z box)] [zz (z box)] [yz (rect)] [b (+1 box)]
// ---------------------------------------------------------------------------
template <int M>
struct VL {
    using B = BX<M>;
    static constexpr int OXY = 0, OYY = B::YS, OXZ = 2 * B::YS, OZZ = OXZ + B::ZS, OYZ = OZZ + B::ZS,
                         OB = OYZ + B::RS, SZ = OB + B::PS;
    static constexpr uint32_t BYTES = 4u * (2 * B::YR * B::YC + 2 * B::ZR * B::ZC + B::RR * B::RC +
                                            B::PR * B::PC);
};

template <int M>
__global__ void __launch_bounds__(NT, 2)
el_vpass_tma(GridDev g, FDW w, F9 s, const float *__restrict__ bu,
             const __grid_constant__ CUtensorMap mxy, const __grid_constant__ CUtensorMap myy,
             const __grid_constant__ CUtensorMap mxz, const __grid_constant__ CUtensorMap mzz,
             const __grid_constant__ CUtensorMap myz, const __grid_constant__ CUtensorMap mb, int xc,
             int *err)
{
    using L = VL<M>;
    using B = BX<M>;
    constexpr int Q = 2 * M;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y;
    const bool lead = tz == 0 && ty == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    const float *txx = s.f[3], *txy = s.f[6], *txz = s.f[7];
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        mbar_expect(&bars[st], L::BYTES);
        tma3(S + L::OXY, &mxy, z0, y0 - M, x, &bars[st]);
        tma3(S + L::OYY, &myy, z0, y0 - M, x, &bars[st]);
        tma3(S + L::OXZ, &mxz, z0 - B::MZ, y0, x, &bars[st]);
        tma3(S + L::OZZ, &mzz, z0 - B::MZ, y0, x, &bars[st]);
        tma3(S + L::OYZ, &myz, z0 - B::MZ, y0 - M, x, &bars[st]);
        tma3(S + L::OB, &mb, z0, y0, x, &bars[st]);
    };
    if (lead) {
        for (int i = 0; i < NSTAGE; i++) mbar_init(&bars[i], 1);
        fence_init();
    }
    __syncthreads();
    if (lead)
        for (int i = 0; i < NSTAGE - 1 && xa + i < xb; i++) issue(xa + i, i);
    const bool act = y < g.NY && z < g.NZ;
    const long long pl = (long long)g.NY * g.NZ;
    const long long q0 = act ? (long long)y * g.NZ + z : 0;
    float qxx[Q], qxy[Q], qxz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        const int xq = xa - M + 1 + j, xr = xa - M + j;
        qxx[j] = act && xq >= 0 && xq < g.NX ? __ldg(txx + xq * pl + q0) : 0.f;
        qxy[j] = act && xr >= 0 && xr < g.NX ? __ldg(txy + xr * pl + q0) : 0.f;
        qxz[j] = act && xr >= 0 && xr < g.NX ? __ldg(txz + xr * pl + q0) : 0.f;
    }
    float nxx = 0.f, nxy = 0.f, nxz = 0.f, nbx = 0.f, nv0 = 0.f, nv1 = 0.f, nv2 = 0.f;
    auto fetch = [&](int x) {
        if (!act) return;
        nxx = x + M < g.NX ? __ldg(txx + (x + M) * pl + q0) : 0.f;
        nxy = x + M - 1 < g.NX ? __ldg(txy + (x + M - 1) * pl + q0) : 0.f;
        nxz = x + M - 1 < g.NX ? __ldg(txz + (x + M - 1) * pl + q0) : 0.f;
        nbx = __ldg(bu + min(x + 1, g.NX - 1) * pl + q0);
        nv0 = s.f[0][x * pl + q0];
        nv1 = s.f[1][x * pl + q0];
        nv2 = s.f[2][x * pl + q0];
    };
    fetch(xa);
    const float c = g.dt * g.ih;
    const float gzn = __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * min(z, g.NZ - 1));
    const float gzh = __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * min(z, g.NZ - 1) + 1);
    const float gyn = __ldg(g.tab + 2 * g.NX + 2 * min(y, g.NY - 1));
    const float gyh = __ldg(g.tab + 2 * g.NX + 2 * min(y, g.NY - 1) + 1);
    const int cy = ty + M, cz = tz + B::MZ;
    for (int x = xa; x < xb; x++) {
        const int it = x - xa;
        qxx[Q - 1] = nxx;
        qxy[Q - 1] = nxy;
        qxz[Q - 1] = nxz;
        const float v0 = nv0, v1 = nv1, v2 = nv2, bxn = nbx;
        // all threads are past iteration it-1: its stage may be refilled
        __syncthreads();
        if (lead && x + NSTAGE - 1 < xb) issue(x + NSTAGE - 1, (it + NSTAGE - 1) % NSTAGE);
        if (x + 1 < xb) fetch(x + 1);
        if (!stage_wait(bars, it, err)) return;
        const float *S = sm + (it % NSTAGE) * L::SZ;
        if (act) {
            const float *sxy = S + L::OXY, *syy = S + L::OYY, *sxz = S + L::OXZ, *szz = S + L::OZZ,
                        *syz = S + L::OYZ, *sb = S + L::OB;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float b = w.b[k - 1];
                d0 += b * ((qxx[M - 1 + k] - qxx[M - k]) +
                           (sxy[(cy + k - 1) * B::YC + tz] - sxy[(cy - k) * B::YC + tz]) +
                           (sxz[ty * B::ZC + cz + k - 1] - sxz[ty * B::ZC + cz - k]));
                d1 += b * ((qxy[M + k - 1] - qxy[M - k]) +
                           (syy[(cy + k) * B::YC + tz] - syy[(cy - k + 1) * B::YC + tz]) +
                           (syz[cy * B::RC + cz + k - 1] - syz[cy * B::RC + cz - k]));
                d2 += b * ((qxz[M + k - 1] - qxz[M - k]) +
                           (syz[(cy + k - 1) * B::RC + cz] - syz[(cy - k) * B::RC + cz]) +
                           (szz[ty * B::ZC + cz + k] - szz[ty * B::ZC + cz - k + 1]));
            }
            const float b0 = sb[ty * B::PC + tz];
            const float bx = 0.5f * (b0 + bxn);
            const float by = 0.5f * (b0 + sb[(y + 1 < g.NY ? ty + 1 : ty) * B::PC + tz]);
            const float bz = 0.5f * (b0 + sb[ty * B::PC + (z + 1 < g.NZ ? tz + 1 : tz)]);
            const float gxn = __ldg(g.tab + 2 * x), gxh = __ldg(g.tab + 2 * x + 1);
            const long long q = x * pl + q0;
            s.f[0][q] = gxh * gyn * gzn * (v0 + c * bx * d0);
            s.f[1][q] = gxn * gyh * gzn * (v1 + c * by * d1);
            s.f[2][q] = gxn * gyn * gzh * (v2 + c * bz * d2);
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
// elastic stress pass
// stage: [vx rect] [vy rect] [vz rect] [mu +1 box, plane x] [mu +1 box, plane x+1]
// ---------------------------------------------------------------------------
template <int M>
struct TL {
    using B = BX<M>;
    static constexpr int OVX = 0, OVY = B::RS, OVZ = 2 * B::RS, OM0 = 3 * B::RS, OM1 = OM0 + B::PS,
                         SZ = OM1 + B::PS;
    static constexpr uint32_t BYTES = 4u * (3 * B::RR * B::RC + 2 * B::PR * B::PC);
};

template <int M>
__global__ void __launch_bounds__(NT, 2)
el_tpass_tma(GridDev g, FDW w, F9 s, const float *__restrict__ lam,
             const __grid_constant__ CUtensorMap mvx, const __grid_constant__ CUtensorMap mvy,
             const __grid_constant__ CUtensorMap mvz, const __grid_constant__ CUtensorMap mmu, int xc,
             int *err)
{
    using L = TL<M>;
    using B = BX<M>;
    constexpr int Q = 2 * M;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y;
    const bool lead = tz == 0 && ty == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    const float *vxp = s.f[0], *vyp = s.f[1], *vzp = s.f[2];
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        mbar_expect(&bars[st], L::BYTES);
        tma3(S + L::OVX, &mvx, z0 - B::MZ, y0 - M, x, &bars[st]);
        tma3(S + L::OVY, &mvy, z0 - B::MZ, y0 - M, x, &bars[st]);
        tma3(S + L::OVZ, &mvz, z0 - B::MZ, y0 - M, x, &bars[st]);
        tma3(S + L::OM0, &mmu, z0, y0, x, &bars[st]);
        tma3(S + L::OM1, &mmu, z0, y0, min(x + 1, g.NX - 1), &bars[st]);
    };
    if (lead) {
        for (int i = 0; i < NSTAGE; i++) mbar_init(&bars[i], 1);
        fence_init();
    }
    __syncthreads();
    if (lead)
        for (int i = 0; i < NSTAGE - 1 && xa + i < xb; i++) issue(xa + i, i);
    const bool act = y < g.NY && z < g.NZ;
    const long long pl = (long long)g.NY * g.NZ;
    const long long q0 = act ? (long long)y * g.NZ + z : 0;
    float qvx[Q], qvy[Q], qvz[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        const int xr = xa - M + j, xq = xa - M + 1 + j;
        qvx[j] = act && xr >= 0 && xr < g.NX ? __ldg(vxp + xr * pl + q0) : 0.f;
        qvy[j] = act && xq >= 0 && xq < g.NX ? __ldg(vyp + xq * pl + q0) : 0.f;
        qvz[j] = act && xq >= 0 && xq < g.NX ? __ldg(vzp + xq * pl + q0) : 0.f;
    }
    float nvx = 0.f, nvy = 0.f, nvz = 0.f;
    auto fetch = [&](int x) {
        if (!act) return;
        nvx = x + M - 1 < g.NX ? __ldg(vxp + (x + M - 1) * pl + q0) : 0.f;
        nvy = x + M < g.NX ? __ldg(vyp + (x + M) * pl + q0) : 0.f;
        nvz = x + M < g.NX ? __ldg(vzp + (x + M) * pl + q0) : 0.f;
    };
    fetch(xa);
    const float c = g.dt * g.ih;
    const int zc = min(z, g.NZ - 1), yc = min(y, g.NY - 1);
    const float gzn = __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * zc),
                gzh = __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * zc + 1);
    const float gyn = __ldg(g.tab + 2 * g.NX + 2 * yc), gyh = __ldg(g.tab + 2 * g.NX + 2 * yc + 1);
    const int cy = ty + M, cz = tz + B::MZ;
    const int y1 = y + 1 < g.NY ? ty + 1 : ty, z1 = z + 1 < g.NZ ? tz + 1 : tz;
    for (int x = xa; x < xb; x++) {
        const int it = x - xa;
        qvx[Q - 1] = nvx;
        qvy[Q - 1] = nvy;
        qvz[Q - 1] = nvz;
        __syncthreads();
        if (lead && x + NSTAGE - 1 < xb) issue(x + NSTAGE - 1, (it + NSTAGE - 1) % NSTAGE);
        const long long q = x * pl + q0;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, t4 = 0.f, t5 = 0.f, l = 0.f;
        if (act) {
            t0 = s.f[3][q]; t1 = s.f[4][q]; t2 = s.f[5][q];
            t3 = s.f[6][q]; t4 = s.f[7][q]; t5 = s.f[8][q];
            l = __ldg(lam + q);
        }
        if (x + 1 < xb) fetch(x + 1);
        if (!stage_wait(bars, it, err)) return;
        const float *S = sm + (it % NSTAGE) * L::SZ;
        if (act) {
            const float *svx = S + L::OVX, *svy = S + L::OVY, *svz = S + L::OVZ;
            float exx = 0.f, eyy = 0.f, ezz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float b = w.b[k - 1];
                exx += b * (qvx[M + k - 1] - qvx[M - k]);
                eyy += b * (svy[(cy + k - 1) * B::RC + cz] - svy[(cy - k) * B::RC + cz]);
                ezz += b * (svz[cy * B::RC + cz + k - 1] - svz[cy * B::RC + cz - k]);
                gxy += b * ((svx[(cy + k) * B::RC + cz] - svx[(cy - k + 1) * B::RC + cz]) +
                            (qvy[M - 1 + k] - qvy[M - k]));
                gxz += b * ((svx[cy * B::RC + cz + k] - svx[cy * B::RC + cz - k + 1]) +
                            (qvz[M - 1 + k] - qvz[M - k]));
                gyz += b * ((svy[cy * B::RC + cz + k] - svy[cy * B::RC + cz - k + 1]) +
                            (svz[(cy + k) * B::RC + cz] - svz[(cy - k + 1) * B::RC + cz]));
            }
            const float *R0 = S + L::OM0, *R1 = S + L::OM1;
            const float m0 = R0[ty * B::PC + tz], my = R0[y1 * B::PC + tz], mz = R0[ty * B::PC + z1];
            const float mx = R1[ty * B::PC + tz], mxy_ = R1[y1 * B::PC + tz], mxz_ = R1[ty * B::PC + z1];
            const float myz_ = R0[y1 * B::PC + z1];
            const float mxy = 0.25f * (m0 + mx + my + mxy_);
            const float mxz = 0.25f * (m0 + mx + mz + mxz_);
            const float myz = 0.25f * (m0 + my + mz + myz_);
            const float tr = exx + eyy + ezz, m2 = 2.f * m0;
            const float gxn = __ldg(g.tab + 2 * x), gxh = __ldg(g.tab + 2 * x + 1);
            const float gn = gxn * gyn * gzn;
            s.f[3][q] = gn * (t0 + c * (l * tr + m2 * exx));
            s.f[4][q] = gn * (t1 + c * (l * tr + m2 * eyy));
            s.f[5][q] = gn * (t2 + c * (l * tr + m2 * ezz));
            s.f[6][q] = gxh * gyh * gzn * (t3 + c * mxy * gxy);
            s.f[7][q] = gxh * gyn * gzh * (t4 + c * mxz * gxz);
            s.f[8][q] = gxn * gyh * gzh * (t5 + c * myz * gyz);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qvx[j] = qvx[j + 1];
            qvy[j] = qvy[j + 1];
            qvz[j] = qvz[j + 1];
        }
    }
}

// ---------------------------------------------------------------------------
// TTI rotation pass.  stage: [p rect] [r rect] (+ [eps rect] [del rect] ADJ)
// ---------------------------------------------------------------------------
template <int M, int ADJ>
struct RL {
    using B = BX<M>;
    static constexpr int OP = 0, OR = B::RS, OE = 2 * B::RS, OD = 3 * B::RS,
                         SZ = (ADJ ? 4 : 2) * B::RS;
    static constexpr uint32_t BYTES = 4u * (ADJ ? 4 : 2) * B::RR * B::RC;
};

template <int M, int ADJ>
__global__ void __launch_bounds__(NT, 2)
tti_rot_tma(GridDev g, FDW w, const float *__restrict__ p, const float *__restrict__ r,
            const float *__restrict__ eps, const float *__restrict__ del,
            const float *__restrict__ th, const float *__restrict__ ph,
            const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap mr,
            const __grid_constant__ CUtensorMap me, const __grid_constant__ CUtensorMap md,
            float *__restrict__ ex, float *__restrict__ ey, float *__restrict__ ez,
            float *__restrict__ fx, float *__restrict__ fy, float *__restrict__ fz, int xc, int *err)
{
    using L = RL<M, ADJ>;
    using B = BX<M>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y, tid = ty * FZ + tz;
    const bool lead = tid == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        mbar_expect(&bars[st], L::BYTES);
        tma3(S + L::OP, &mp, z0 - B::MZ, y0 - M, x, &bars[st]);
        tma3(S + L::OR, &mr, z0 - B::MZ, y0 - M, x, &bars[st]);
        if (ADJ) {
            tma3(S + L::OE, &me, z0 - B::MZ, y0 - M, x, &bars[st]);
            tma3(S + L::OD, &md, z0 - B::MZ, y0 - M, x, &bars[st]);
        }
    };
    if (lead) {
        for (int i = 0; i < NSTAGE; i++) mbar_init(&bars[i], 1);
        fence_init();
    }
    __syncthreads();
    if (lead)
        for (int i = 0; i < NSTAGE - 1 && xa + i < xb; i++) issue(xa + i, i);
    const bool act = y < g.NY && z < g.NZ;
    const long long pl = (long long)g.NY * g.NZ;
    const long long q0 = act ? (long long)y * g.NZ + z : 0;
    // (p, r) or zeta = C (lam_p, lam_r) at own column, plane x
    auto own = [&](int x, float &a, float &b) {
        a = b = 0.f;
        if (!act || x < 0 || x >= g.NX) return;
        const long long q = x * pl + q0;
        const float u = __ldg(p + q), v = __ldg(r + q);
        if (!ADJ) { a = u; b = v; return; }
        const float c1 = 1.f + 2.f * __ldg(eps + q), c2 = sqrtf(1.f + 2.f * __ldg(del + q));
        a = c1 * u + c2 * v;
        b = c2 * u + v;
    };
    float qp[Q], qr[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) own(xa - M + j, qp[j], qr[j]);
    float np_ = 0.f, nr_ = 0.f, nth = 0.f, nph = 0.f;
    auto fetch = [&](int x) {
        own(x + M, np_, nr_);
        if (act) {
            nth = __ldg(th + x * pl + q0);
            nph = __ldg(ph + x * pl + q0);
        }
    };
    fetch(xa);
    const int cy = ty + M, cz = tz + B::MZ;
    const int ci = cy * B::RC + cz;
    for (int x = xa; x < xb; x++) {
        const int it = x - xa;
        qp[Q - 1] = np_;
        qr[Q - 1] = nr_;
        const float th_ = nth, ph_ = nph;
        __syncthreads();
        if (lead && x + NSTAGE - 1 < xb) issue(x + NSTAGE - 1, (it + NSTAGE - 1) % NSTAGE);
        if (x + 1 < xb) fetch(x + 1);
        if (!stage_wait(bars, it, err)) return;
        float *S = sm + (it % NSTAGE) * L::SZ;
        if (ADJ) {
            // zeta = C lam over the whole rectangle, in place (each thread a share)
            float *sp = S + L::OP, *sr = S + L::OR;
            const float *se = S + L::OE, *sd = S + L::OD;
            for (int i = tid; i < B::RR * B::RC; i += NT) {
                const float c1 = 1.f + 2.f * se[i], c2 = sqrtf(1.f + 2.f * sd[i]);
                const float u = sp[i], v = sr[i];
                sp[i] = c1 * u + c2 * v;
                sr[i] = c2 * u + v;
            }
            __syncthreads();
        }
        if (act) {
            const float *sp = S + L::OP, *sr = S + L::OR;
            float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f, gr0 = 0.f, gr1 = 0.f, gr2 = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                gp0 += c * (qp[M + k] - qp[M - k]);
                gr0 += c * (qr[M + k] - qr[M - k]);
                gp1 += c * (sp[ci + k * B::RC] - sp[ci - k * B::RC]);
                gr1 += c * (sr[ci + k * B::RC] - sr[ci - k * B::RC]);
                gp2 += c * (sp[ci + k] - sp[ci - k]);
                gr2 += c * (sr[ci + k] - sr[ci - k]);
            }
            float st, ct, sph, cph;
            sincosf(th_, &st, &ct);
            sincosf(ph_, &sph, &cph);
            const float n0 = st * cph, n1 = st * sph, n2 = ct;
            gp0 *= g.ih; gp1 *= g.ih; gp2 *= g.ih;
            gr0 *= g.ih; gr1 *= g.ih; gr2 *= g.ih;
            const float wp = n0 * gp0 + n1 * gp1 + n2 * gp2;
            const float wr = n0 * gr0 + n1 * gr1 + n2 * gr2;
            const long long q = x * pl + q0;
            ex[q] = gp0 - n0 * wp;
            ey[q] = gp1 - n1 * wp;
            ez[q] = gp2 - n2 * wp;
            fx[q] = n0 * wr;
            fy[q] = n1 * wr;
            fz[q] = n2 * wr;
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qp[j] = qp[j + 1];
            qr[j] = qr[j + 1];
        }
    }
}

// ---------------------------------------------------------------------------
// TTI update pass.  stage: [e_y y box] [f_y y box] [e_z z box] [f_z z box]
// ---------------------------------------------------------------------------
template <int M>
struct UL {
    using B = BX<M>;
    static constexpr int OEY = 0, OFY = B::YS, OEZ = 2 * B::YS, OFZ = OEZ + B::ZS, SZ = OFZ + B::ZS;
    static constexpr uint32_t BYTES = 4u * (2 * B::YR * B::YC + 2 * B::ZR * B::ZC);
};

template <int M, int ADJ>
__global__ void __launch_bounds__(NT, 2)
tti_upd_tma(GridDev g, FDW w, const float *__restrict__ ex, const float *__restrict__ fx,
            const __grid_constant__ CUtensorMap mey, const __grid_constant__ CUtensorMap mfy,
            const __grid_constant__ CUtensorMap mez, const __grid_constant__ CUtensorMap mfz,
            const float *__restrict__ m, const float *__restrict__ eps, const float *__restrict__ del,
            const float *__restrict__ pc, const float *__restrict__ rc, float *__restrict__ pp,
            float *__restrict__ rp, const float *__restrict__ up, const float *__restrict__ ur,
            float *__restrict__ grad, int *flag, int check, int xc, int *err)
{
    using L = UL<M>;
    using B = BX<M>;
    constexpr int Q = 2 * M + 1;
    extern __shared__ __align__(128) float sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NSTAGE * L::SZ);   // after the ring
    const int tz = threadIdx.x, ty = threadIdx.y;
    const bool lead = tz == 0 && ty == 0;
    const int z0 = blockIdx.x * FZ, y0 = blockIdx.y * FY;
    const int z = z0 + tz, y = y0 + ty;
    const int xa = blockIdx.z * xc, xb = min(xa + xc, g.NX);
    auto issue = [&](int x, int st) {
        float *S = sm + st * L::SZ;
        mbar_expect(&bars[st], L::BYTES);
        tma3(S + L::OEY, &mey, z0, y0 - M, x, &bars[st]);
        tma3(S + L::OFY, &mfy, z0, y0 - M, x, &bars[st]);
        tma3(S + L::OEZ, &mez, z0 - B::MZ, y0, x, &bars[st]);
        tma3(S + L::OFZ, &mfz, z0 - B::MZ, y0, x, &bars[st]);
    };
    if (lead) {
        for (int i = 0; i < NSTAGE; i++) mbar_init(&bars[i], 1);
        fence_init();
    }
    __syncthreads();
    if (lead)
        for (int i = 0; i < NSTAGE - 1 && xa + i < xb; i++) issue(xa + i, i);
    const bool act = y < g.NY && z < g.NZ;
    const long long pl = (long long)g.NY * g.NZ;
    const long long q0 = act ? (long long)y * g.NZ + z : 0;
    float qe[Q], qf[Q];
#pragma unroll
    for (int j = 0; j < Q - 1; j++) {
        const int xq = xa - M + j;
        const bool in = act && xq >= 0 && xq < g.NX;
        qe[j] = in ? __ldg(ex + xq * pl + q0) : 0.f;
        qf[j] = in ? __ldg(fx + xq * pl + q0) : 0.f;
    }
    float ne = 0.f, nf = 0.f;
    auto fetch = [&](int x) {
        const bool in = act && x + M < g.NX;
        ne = in ? __ldg(ex + (x + M) * pl + q0) : 0.f;
        nf = in ? __ldg(fx + (x + M) * pl + q0) : 0.f;
    };
    fetch(xa);
    const float *sx = g.tab, *sy = g.tab + g.NX, *sz = g.tab + g.NX + g.NY;
    const float dt2 = g.dt * g.dt, hdt = 0.5f * g.dt;
    const float syz = act ? __ldg(sy + y) + __ldg(sz + z) : 0.f;
    const int iy = (ty + M) * B::YC + tz, iz = ty * B::ZC + tz + B::MZ;
    for (int x = xa; x < xb; x++) {
        const int it = x - xa;
        qe[Q - 1] = ne;
        qf[Q - 1] = nf;
        __syncthreads();
        if (lead && x + NSTAGE - 1 < xb) issue(x + NSTAGE - 1, (it + NSTAGE - 1) % NSTAGE);
        const long long q = x * pl + q0;
        float mm = 1.f, e_ = 0.f, d_ = 0.f, p1 = 0.f, r1 = 0.f, p0 = 0.f, r0 = 0.f;
        if (act) {
            mm = __ldg(m + q);
            if (!ADJ) {
                e_ = __ldg(eps + q);
                d_ = __ldg(del + q);
            }
            p1 = __ldg(pc + q);
            r1 = __ldg(rc + q);
            p0 = pp[q];
            r0 = rp[q];
        }
        if (x + 1 < xb) fetch(x + 1);
        if (!stage_wait(bars, it, err)) return;
        const float *S = sm + (it % NSTAGE) * L::SZ;
        if (act) {
            const float *sey = S + L::OEY, *sfy = S + L::OFY, *sez = S + L::OEZ, *sfz = S + L::OFZ;
            float h0 = 0.f, hz = 0.f;
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float c = w.c[k - 1];
                h0 += c * ((qe[M + k] - qe[M - k]) + (sey[iy + k * B::YC] - sey[iy - k * B::YC]) +
                           (sez[iz + k] - sez[iz - k]));
                hz += c * ((qf[M + k] - qf[M - k]) + (sfy[iy + k * B::YC] - sfy[iy - k * B::YC]) +
                           (sfz[iz + k] - sfz[iz - k]));
            }
            h0 *= g.ih;
            hz *= g.ih;
            float Lp, Lr;
            if (!ADJ) {
                const float a = 1.f + 2.f * e_, s2 = sqrtf(1.f + 2.f * d_);
                Lp = a * h0 + s2 * hz;
                Lr = s2 * h0 + hz;
            } else {
                Lp = h0;
                Lr = hz;
            }
            const float sd = hdt * (__ldg(sx + x) + syz);
            const float A = mm * (1.f + sd), Bc = mm * (1.f - sd);
            const float pn = (dt2 * Lp + 2.f * mm * p1 - Bc * p0) / A;
            const float rn = (dt2 * Lr + 2.f * mm * r1 - Bc * r0) / A;
            pp[q] = pn;
            rp[q] = rn;
            if (ADJ && grad) grad[q] -= dt2 * (__ldg(up + q) * Lp + __ldg(ur + q) * Lr) / mm;
            if (check && !(isfinite(pn) && isfinite(rn))) atomicOr(flag, 1);
        }
#pragma unroll
        for (int j = 0; j < Q - 1; j++) {
            qe[j] = qe[j + 1];
            qf[j] = qf[j + 1];
        }
    }
}

// ---------------------------------------------------------------------------
// host: tensor maps
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)f;
    });
    return fn;
}

// 3D map of a [NX][NY][NZ] float array, box (bz, by, 1); zero fill outside
bool make_map(CUtensorMap *m, const float *base, const GridDev &g, int bz, int by)
{
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.NZ, (cuuint64_t)g.NY, (cuuint64_t)g.NX};
    cuuint64_t strides[2] = {(cuuint64_t)g.NZ * 4, (cuuint64_t)g.NZ * g.NY * 4};
    cuuint32_t box[3] = {(cuuint32_t)bz, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class K>
void set_smem(K kernel, size_t bytes)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int M>
int el_launch(prop_s *P, float *const *S, float dt)
{
    using B = BX<M>;
    GridDev g = P->g;
    g.dt = dt;
    const int xc = P->xchunk;
    dim3 blk(FZ, FY, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    F9 s;
    for (int i = 0; i < 9; i++) s.f[i] = S[i];
    CUtensorMap mxy, myy, mxz, mzz, myz, mb, mvx, mvy, mvz, mmu;
    bool ok = make_map(&mxy, S[6], g, B::YC, B::YR) && make_map(&myy, S[4], g, B::YC, B::YR) &&
              make_map(&mxz, S[7], g, B::ZC, B::ZR) && make_map(&mzz, S[5], g, B::ZC, B::ZR) &&
              make_map(&myz, S[8], g, B::RC, B::RR) && make_map(&mb, P->bu, g, B::PC, B::PR) &&
              make_map(&mvx, S[0], g, B::RC, B::RR) && make_map(&mvy, S[1], g, B::RC, B::RR) &&
              make_map(&mvz, S[2], g, B::RC, B::RR) && make_map(&mmu, P->mu, g, B::PC, B::PR);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = NSTAGE * VL<M>::SZ * sizeof(float) + 64, s2 = NSTAGE * TL<M>::SZ * sizeof(float) + 64;
    static const bool attr = (set_smem(el_vpass_tma<M>, s1), set_smem(el_tpass_tma<M>, s2), true);
    (void)attr;
    el_vpass_tma<M><<<grd, blk, s1, P->stream>>>(g, P->w, s, P->bu, mxy, myy, mxz, mzz, myz, mb, xc, P->flag);
    el_tpass_tma<M><<<grd, blk, s2, P->stream>>>(g, P->w, s, P->lam, mvx, mvy, mvz, mmu, xc, P->flag);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

template <int M, int ADJ>
int tti_launch(prop_s *P, float *const *S, const float *up, const float *ur, float *grad)
{
    using B = BX<M>;
    const GridDev &g = P->g;
    const int xc = P->xchunk;
    dim3 blk(FZ, FY, 1), grd((g.NZ + FZ - 1) / FZ, (g.NY + FY - 1) / FY, (g.NX + xc - 1) / xc);
    float *const *t = P->tmp;
    CUtensorMap mp, mr, me, md, mey, mfy, mez, mfz;
    bool ok = make_map(&mp, S[0], g, B::RC, B::RR) && make_map(&mr, S[1], g, B::RC, B::RR) &&
              make_map(&me, P->eps, g, B::RC, B::RR) && make_map(&md, P->del, g, B::RC, B::RR) &&
              make_map(&mey, t[1], g, B::YC, B::YR) && make_map(&mfy, t[4], g, B::YC, B::YR) &&
              make_map(&mez, t[2], g, B::ZC, B::ZR) && make_map(&mfz, t[5], g, B::ZC, B::ZR);
    if (!ok) return wp_fail(P, PROP_ECUDA, "cuTensorMapEncodeTiled failed");
    const size_t s1 = NSTAGE * RL<M, ADJ>::SZ * sizeof(float) + 64,
                 s2 = NSTAGE * UL<M>::SZ * sizeof(float) + 64;
    static const bool attr = (set_smem(tti_rot_tma<M, ADJ>, s1), set_smem(tti_upd_tma<M, ADJ>, s2), true);
    (void)attr;
    tti_rot_tma<M, ADJ><<<grd, blk, s1, P->stream>>>(g, P->w, S[0], S[1], P->eps, P->del, P->th, P->ph, mp, mr,
                                                    me, md, t[0], t[1], t[2], t[3], t[4], t[5], xc, P->flag);
    tti_upd_tma<M, ADJ><<<grd, blk, s2, P->stream>>>(g, P->w, t[0], t[3], mey, mfy, mez, mfz, P->m, P->eps,
                                                    P->del, S[0], S[1], S[2], S[3], up, ur, grad, P->flag,
                                                    P->d.check_nan, xc, P->flag);
    P->kern_launches += 2;
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

}  // namespace

// TMA-fed passes need 16-byte row strides (NZ a multiple of 4) and the
// driver's tensor-map encoder
bool tma_usable(const prop_s *P)
{
    return P->g.NZ % 4 == 0 && encode_fn() != nullptr && getenv("WAVEPROP_NO_TMA") == nullptr;
}

// elastic step with time step dt_sign * dt (forward: +1; adjoint modelling
// in (b_avg vbar, g C tbar) variables: -1)
int el_launch_tma(prop_s *P, float *const *S, float dt_sign)
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

int tti_launch_tma(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                   float *grad)
{
    prof_begin(P, adjoint ? 1 : 0);
    int rc;
    switch (P->M) {
    case 2: rc = adjoint ? tti_launch<2, 1>(P, S, img_p, img_r, grad) : tti_launch<2, 0>(P, S, img_p, img_r, grad); break;
    case 4: rc = adjoint ? tti_launch<4, 1>(P, S, img_p, img_r, grad) : tti_launch<4, 0>(P, S, img_p, img_r, grad); break;
    case 6: rc = adjoint ? tti_launch<6, 1>(P, S, img_p, img_r, grad) : tti_launch<6, 0>(P, S, img_p, img_r, grad); break;
    case 8: rc = adjoint ? tti_launch<8, 1>(P, S, img_p, img_r, grad) : tti_launch<8, 0>(P, S, img_p, img_r, grad); break;
    default: return wp_fail(P, PROP_EINVAL, "unsupported space order");
    }
    prof_end(P, adjoint ? 1 : 0);
    return rc;
}
