// TMA plane-ring machinery shared by the TMA-fed stencil passes: tile
// geometry (32 z x FY y columns, two z points per consumer thread, one
// producer warp), mbarrier and cp.async.bulk.tensor helpers in inline PTX,
// the bounded producer/consumer ring, and the host side that encodes
// (and caches per handle) the 3D tensor maps.
//
// The tile height FY is a compile-time constant of the translation unit
// (WP_TILE_Y: 8, 16 or 32 rows; 16 unless the unit defines it).  The
// stencil passes are compiled once per height and the autotuner picks one
// per grid; the arithmetic of a point does not depend on the tile, so every
// height gives the same bits.
#pragma once
#include "tile.cuh"

#include <cuda.h>
#include <cstdlib>
#include <mutex>

#ifndef WP_TILE_Y
#define WP_TILE_Y 16
#endif
static_assert(WP_TILE_Y == 8 || WP_TILE_Y == 16 || WP_TILE_Y == 32, "tile height must be 8, 16 or 32");

namespace {

constexpr int FY = WP_TILE_Y;
using tile::FZ;

constexpr int TZ2 = FZ / 2;        // threads along z, two points each
constexpr int NT2 = TZ2 * FY;      // consumer threads per CTA (FY / 2 warps)
constexpr int NTP = NT2 + 32;      // + one producer warp
// resident CTAs per SM for the launch bounds: `base` at 16 rows, scaled
// with the CTA size (a 32-row CTA has the threads of two 16-row ones)
constexpr int occ(int base) { return FY == 8 ? 2 * base : (FY == 32 ? 1 : base); }
// Elastic passes above space order 8 need more than 96 registers per thread
// and more shared memory than two CTAs per SM allow: they run one CTA per SM.
constexpr int NSTAGE = 3;

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
#ifdef WP_CHECK
WP_DEV bool ck_tma(const float *dst, int c0);
#endif
WP_DEV void tma3(float *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
#ifdef WP_CHECK
    if (!ck_tma(dst, c0)) return;
#endif
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
WP_DEV void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
// producer after an abort: wait (bounded) for the stages of iterations
// [a, b] that may still be in flight, so no copy lands after the CTA exits
template <int NS = NSTAGE>
WP_DEV void drain(uint64_t *full, int a, int b)
{
    for (int j = a < 0 ? 0 : a; j <= b; j++) mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1));
}

// 8-byte accesses (z even, NZ even: always aligned)
// Bounds-checking build (WP_CHECK, selected at run time by WAVEPROP_CHECK=1):
// every shared-memory read must lie in the CTA's dynamic shared memory, every
// global float2 access of a field below the grid size and every TMA copy
// start on a 16-byte boundary in x and in shared memory.  A failing access is
// skipped (loads return zeros) and bit 8 of the handle's error word is set,
// which the host reports as PROP_ECUDA; nothing traps, and a skipped copy
// ends in the bounded wait of its stage (bit 2).  In the normal build the
// checks compile to nothing.
#ifdef WP_CHECK
static __shared__ unsigned long long wp_ck_n;   // elements of a field
static __shared__ int *wp_ck_err;
extern __shared__ __align__(128) float wp_dsm[];
WP_DEV void ck_begin(unsigned long long n, int *err)
{
    wp_ck_n = n;
    wp_ck_err = err;
}
WP_DEV bool ck_fail()
{
    atomicOr(wp_ck_err, 8);
    return false;
}
WP_DEV bool ck_smem(const void *p, unsigned bytes)
{
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t a = saddr(p), b = saddr(wp_dsm);
    return (a >= b && a + bytes <= b + dyn && (a & (bytes - 1)) == 0) || ck_fail();
}
WP_DEV bool ck_field(unsigned o) { return (unsigned long long)o + 2 <= wp_ck_n || ck_fail(); }
// x (innermost, z) coordinate of a copy: 16-byte multiple; destination
// 16-byte aligned inside the dynamic shared memory
WP_DEV bool ck_tma(const float *dst, int c0) { return ((c0 & 3) == 0 || ck_fail()) && ck_smem(dst, 16); }
#else
WP_DEV void ck_begin(unsigned long long, int *) {}
#endif

WP_DEV float2 lds2(const float *p)
{
#ifdef WP_CHECK
    if (!ck_smem(p, 8)) return make_float2(0.f, 0.f);
#endif
    return *reinterpret_cast<const float2 *>(p);
}
WP_DEV float2 ldg2(const float *__restrict__ p, unsigned o)
{
#ifdef WP_CHECK
    if (!ck_field(o)) return make_float2(0.f, 0.f);
#endif
    return __ldg(reinterpret_cast<const float2 *>(p + o));
}
WP_DEV void st2(float *p, unsigned o, float a, float b)
{
#ifdef WP_CHECK
    if (!ck_field(o)) return;
#endif
    *reinterpret_cast<float2 *>(p + o) = make_float2(a, b);
}
WP_DEV float2 dif2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// paired FP32 arithmetic (one instruction for both lanes; per component the
// result of the scalar operation)
WP_DEV float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
WP_DEV float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
WP_DEV float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
WP_DEV float2 f2s(float a) { return make_float2(a, a); }
// a - b as fma(-1, b, a): the same rounding as the subtraction
WP_DEV float2 f2sub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }

constexpr int al32(int n) { return (n + 31) & ~31; }   // 128-byte aligned float offsets
constexpr int IS = FZ * FY;                             // interior box (tile of one plane)

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

// z window of 2M+2 values starting M before the thread's first point:
// w[M + d] = f(z + d), d = -M .. M+1
template <int M>
WP_DEV void zwin(const float *row, int cz, float (&w)[2 * M + 2])
{
#pragma unroll
    for (int j = 0; j <= M; j++) {
        const float2 a = lds2(row + cz - M + 2 * j);
        w[2 * j] = a.x;
        w[2 * j + 1] = a.y;
    }
}

// Producer/consumer plane ring.  full[s] completes when the copies of a
// stage have landed (one arrive with the byte count + the TMA bytes);
// empty[s] when every consumer warp has finished reading it (one arrive per
// warp).  A dedicated producer warp (its lane 0) keeps NS planes in
// flight: it refills a stage as soon as it is released, so consumers never
// wait for each other.  All waits are bounded; a warp that gives up reports
// bit 2 and leaves, and the producer drains its copies in flight first.
constexpr int NWARP = NT2 / 32;

template <int NS = NSTAGE>
struct RingN {
    uint64_t *full, *empty;
    int st = 0;
    uint32_t ph = 0;
    WP_DEV explicit RingN(uint64_t *bars) : full(bars), empty(bars + NS) {}
    WP_DEV void init()
    {
        for (int i = 0; i < NS; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NWARP);
        }
        fence_init();
    }
    // producer (lane 0 of the producer warp): plane xa + it into stage it % NS
    template <class F>
    WP_DEV void produce(int xa, int nit, F issue, int *err)
    {
        for (int it = 0; it < nit; it++) {
            const int s = it % NS;
            if (it >= NS && !mbar_wait(&empty[s], (uint32_t)(((it / NS) - 1) & 1))) {
                atomicOr(err, 2);
                drain<NS>(full, it - NS, it - 1);
                return;
            }
            issue(xa + it, s);
        }
        // stay until the last copies have landed (bounded), so none can
        // arrive after the CTA has exited even if the consumers gave up
        drain<NS>(full, nit - NS, nit - 1);
    }
    WP_DEV bool wait_full() { return mbar_wait(&full[st], ph); }
    // end of iteration: this warp is done with the stage
    WP_DEV void release(int lane)
    {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (++st == NS) {
            st = 0;
            ph ^= 1u;
        }
    }
};
using Ring = RingN<>;


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

// descriptor of (array, box) from the handle's cache; false if encoding failed
bool map_of(prop_s *P, const float *base, int bz, int by, CUtensorMap *out)
{
    const auto key = std::make_tuple((const void *)base, bz, by);
    auto it = P->tmaps.find(key);
    if (it == P->tmaps.end()) {
        CUtensorMap m;
        if (!make_map(&m, base, P->g, bz, by)) return false;
        it = P->tmaps.emplace(key, m).first;
    }
    *out = it->second;
    return true;
}

template <class K>
bool set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

}  // namespace
