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

// TTI damping rate at a node: sum over axes of sig0 * (d/L)^2, L = nbl*h.
WP_DEV float tti_sigma(const GridDev &g, int x, int y, int z)
{
    if (g.nbl <= 0) return 0.f;
    float inv = 1.f / (float)g.nbl;
    float dx = layer_depth((float)x, g.nbl, g.px) * inv;
    float dy = layer_depth((float)y, g.nbl, g.py) * inv;
    float dz = layer_depth((float)z, g.nbl, g.pz) * inv;
    return g.sig0 * (dx * dx + dy * dy + dz * dz);
}

// Cerjan taper exp(-(a d)^2) per axis at continuous position (sx, sy, sz).
WP_DEV float cerjan(const GridDev &g, float sx, float sy, float sz)
{
    if (g.nbl <= 0) return 1.f;
    float dx = g.cer * layer_depth(sx, g.nbl, g.px);
    float dy = g.cer * layer_depth(sy, g.nbl, g.py);
    float dz = g.cer * layer_depth(sz, g.nbl, g.pz);
    return expf(-(dx * dx + dy * dy + dz * dz));
}

// load with zero extension outside the computational grid
WP_DEV float ldz(const float *__restrict__ f, const GridDev &g, int x, int y, int z)
{
    return (x >= 0 && x < g.NX && y >= 0 && y < g.NY && z >= 0 && z < g.NZ) ? __ldg(f + gidx(g, x, y, z)) : 0.f;
}

WP_DEV int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
