// Device helpers shared by the waveprop kernels.
#pragma once
#include "internal.h"

#define WP_DEV __device__ __forceinline__

WP_DEV long long gidx(const GridDev &g, int x, int y, int z)
{
    return ((long long)x * g.NY + y) * g.NZ + z;
}

// depth (cells, continuous) of coordinate s into the absorbing layer of an
// axis with physical points [nbl, nbl + n - 1]
WP_DEV float layer_depth(float s, int nbl, int n)
{
    float lo = (float)nbl, hi = (float)(nbl + n - 1);
    return s < lo ? lo - s : (s > hi ? s - hi : 0.f);
}

// TTI damping rate at a node: sum over axes of sig0 * (d/L)^2, L = nbl*h
// (per-axis table).
WP_DEV float tti_sigma(const GridDev &g, int x, int y, int z)
{
    return __ldg(g.tab + x) + __ldg(g.tab + g.NX + y) + __ldg(g.tab + g.NX + g.NY + z);
}

// Cerjan taper: product over axes of exp(-(0.015 d)^2) at the position
// (sx, sy, sz), each coordinate a node i or a half point i + 1/2 (table).
WP_DEV float cerjan(const GridDev &g, float sx, float sy, float sz)
{
    const int ix = (int)sx, iy = (int)sy, iz = (int)sz;
    const int hx = (sx - ix) > 0.25f, hy = (sy - iy) > 0.25f, hz = (sz - iz) > 0.25f;
    return __ldg(g.tab + 2 * ix + hx) * __ldg(g.tab + 2 * g.NX + 2 * iy + hy) *
           __ldg(g.tab + 2 * (g.NX + g.NY) + 2 * iz + hz);
}

// load with zero extension outside the computational grid
WP_DEV float ldz(const float *__restrict__ f, const GridDev &g, int x, int y, int z)
{
    return (x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ) ? __ldg(f + gidx(g, x, y, z)) : 0.f;
}

WP_DEV int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
