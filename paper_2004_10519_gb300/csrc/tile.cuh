// Tile machinery shared by the pipelined stencil passes: a CTA owns an
// FZ x FY tile of (y, z) columns and streams along x; shared planes with an
// M-cell halo in y and/or z; halo elements are spread evenly over the
// threads (HaloShare) so that every thread issues the same number of loads.
#pragma once
#include "common.cuh"

namespace tile {

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

}  // namespace tile
