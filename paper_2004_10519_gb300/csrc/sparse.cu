// Sparse operators (source injection, receiver interpolation; Sec. II-A:
// s.inject(u.forward, expr=s*dt**2/m) and d.interpolate(u)), model set-up,
// gradient fold, reductions and the snapshot codec.
#include "common.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <tuple>

namespace {
constexpr int NB = 256;

inline int nblk(long long n, int b = NB) { return (int)std::min<long long>((n + b - 1) / b, 1 << 30); }

// tdev != NULL: the time index comes from device memory (steps replayed from
// a CUDA graph) and `out` is the base of the [nt][n] staging array
__global__ void record_kernel(int n, const long long *__restrict__ idx, const float *__restrict__ w,
                              const float *__restrict__ f0, const float *__restrict__ f1,
                              const float *__restrict__ f2, float scale, float *__restrict__ out,
                              const int *__restrict__ tdev)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (tdev) out += (long long)(*tdev) * n;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const long long q = idx[8 * i + c];
        const float wc = w[8 * i + c];
        if (wc != 0.f) {
            float v = f0[q];
            if (f1) v += f1[q];
            if (f2) v += f2[q];
            s += wc * v;
        }
    }
    out[i] = scale * s;
}

__global__ void inject_kernel(GridDev g, int ncell, const long long *__restrict__ cell,
                              const int *__restrict__ ptr, const int *__restrict__ tr,
                              const float *__restrict__ w, const float *__restrict__ traces, int nt,
                              int t, float scale, int mode, const float *__restrict__ m,
                              const float *__restrict__ lam, const float *__restrict__ mu,
                              float *f0, float *f1, float *f2, const float *__restrict__ gu,
                              float *grad, const int *__restrict__ tdev)
{
    // lam, mu: the elastic Lame parameters; for TTI (mode 3) epsilon, delta
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncell) return;
    if (tdev) t = *tdev;
    float acc = 0.f;
    for (int e = ptr[j]; e < ptr[j + 1]; e++) acc += w[e] * traces[(long long)tr[e] * nt + t];
    const long long q = cell[j];
    float coef = scale;
    if (mode == 1 || mode == 3) {
        const int z = (int)(q % g.NZ), y = (int)((q / g.NZ) % g.NY), x = (int)(q / ((long long)g.NZ * g.NY));
        const float A = m[q] * (1.f + 0.5f * tti_sigma(g, x, y, z) * g.dt);
        coef = scale / A;
    } else if (mode == 2 || mode == 4) {
        // residual into u = g C tbar: g (3 lambda + 2 mu) on each diagonal
        // component (mode 4, the x-z plane: g (2 lambda + 2 mu) on xx, zz)
        const int z = (int)(q % g.NZ), y = (int)((q / g.NZ) % g.NY), x = (int)(q / ((long long)g.NZ * g.NY));
        const float gn = g.tab[2 * x] * g.tab[2 * g.NX + 2 * y] * g.tab[2 * (g.NX + g.NY) + 2 * z];
        coef = scale * ((mode == 2 ? 3.f : 2.f) * lam[q] + 2.f * mu[q]) * gn;
    }
    const float v = coef * acc;
    f0[q] += v;
    if (mode == 3) {
        // TTI transposed step: the residual enters lam_p; keep zeta = C lam
        // (f1, f2) consistent: zeta_p += (1 + 2 eps) v, zeta_r += sqrt(1 + 2 delta) v
        f1[q] += (1.f + 2.f * lam[q]) * v;
        f2[q] += sqrtf(1.f + 2.f * mu[q]) * v;
    } else {
        if (f1) f1[q] += v;
        if (f2) f2[q] += v;
    }
    if (grad) grad[q] -= gu[q] * (scale * acc) / m[q];
}

__global__ void record_s_kernel(GridDev g, int n, const long long *__restrict__ idx, const float *__restrict__ w,
                                const float *__restrict__ f0, const float *__restrict__ f1,
                                const float *__restrict__ f2, const float *__restrict__ lam,
                                const float *__restrict__ mu, float nl, float scale, float *__restrict__ out)
{
    // nl = 3 (3D) or 2 (x-z plane, f2 == NULL): C of the unit diagonal is (nl lambda + 2 mu)
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const long long q = idx[8 * i + c];
        const float wc = w[8 * i + c];
        if (wc != 0.f) {
            // tr(tbar) = tr(u) / (g (3 lambda + 2 mu)) at a node
            const int z = (int)(q % g.NZ), y = (int)((q / g.NZ) % g.NY),
                      x = (int)(q / ((long long)g.NZ * g.NY));
            const float gn = g.tab[2 * x] * g.tab[2 * g.NX + 2 * y] * g.tab[2 * (g.NX + g.NY) + 2 * z];
            s += wc * (f0[q] + f1[q] + (f2 ? f2[q] : 0.f)) / ((nl * lam[q] + 2.f * mu[q]) * gn);
        }
    }
    out[i] = scale * s;
}

__global__ void transpose_kernel(const float *__restrict__ in, float *__restrict__ out, int n, int nt)
{
    __shared__ float tile[32][33];
    int t0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int t = t0 + r, i = i0 + threadIdx.x;
        if (t < nt && i < n) tile[r][threadIdx.x] = in[(long long)t * n + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = i0 + r, t = t0 + threadIdx.x;
        if (t < nt && i < n) out[(long long)i * nt + t] = tile[threadIdx.x][r];
    }
}

// mode 0: comp = scale*phys ; 1: comp = 1/(scale*phys)^2
__global__ void extend_kernel(GridDev g, const float *__restrict__ phys, float *__restrict__ comp,
                              float scale, int mode)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= g.N) return;
    const int z = (int)(q % g.NZ), y = (int)((q / g.NZ) % g.NY), x = (int)(q / ((long long)g.NZ * g.NY));
    const int i = clampi(x - g.nbl, 0, g.px - 1), j = clampi(y - g.nby, 0, g.py - 1),
              k = clampi(z - g.nbl, 0, g.pz - 1);
    const float v = phys[((long long)i * g.py + j) * g.pz + k];
    if (mode == 0) comp[q] = scale * v;
    else {
        const float s = scale * v;
        comp[q] = 1.f / (s * s);
    }
}

// elastic: (vp, vs, rho) computational -> (b, lambda, mu) in place
__global__ void lame_kernel(long long n, float *vp_b, float *vs_l, float *rho_mu)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float vp = 1000.f * vp_b[q], vs = 1000.f * vs_l[q], rho = 1000.f * rho_mu[q];
    vp_b[q] = 1.f / rho;
    vs_l[q] = rho * (vp * vp - 2.f * vs * vs);
    rho_mu[q] = rho * vs * vs;
}

// TTI symmetry axis n = (sin th cos ph, sin th sin ph, cos th) (Sec. III-A),
// stored as (n_x, n_y) with the sign flipped where cos th < 0 so that
// n_z = sqrt(1 - n_x^2 - n_y^2); evaluated in double once per model
__global__ void normals_kernel(long long n, const float *th, const float *ph, float *nx, float *ny)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    double st, ct, sp, cp;
    sincos((double)th[q], &st, &ct);
    sincos((double)ph[q], &sp, &cp);
    const double sg = ct < 0.0 ? -1.0 : 1.0;
    nx[q] = (float)(sg * st * cp);
    ny[q] = (float)(sg * st * sp);
}

// adjoint of the edge-replication extension (gather form)
// adjoint of the edge-replication extension along one axis of a [d0][d1][d2]
// array: physical index c of that axis (n points) receives the
// computational cells c + nbl, plus the whole layer in front of c = 0 and
// behind c = n - 1.  Folding the three axes in turn is the transpose of the
// three-axis extension, with at most nbl + 1 terms per output.
__global__ void fold_axis_kernel(const float *__restrict__ in, float *__restrict__ out, int d0, int d1,
                                 int d2, int axis, int n, int nbl)
{
    const int o0 = axis == 0 ? n : d0, o1 = axis == 1 ? n : d1, o2 = axis == 2 ? n : d2;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)o0 * o1 * o2) return;
    const int k = (int)(q % o2), j = (int)((q / o2) % o1), i = (int)(q / ((long long)o2 * o1));
    const int c = axis == 0 ? i : (axis == 1 ? j : k), N = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
    const int lo = c == 0 ? 0 : c + nbl, hi = c == n - 1 ? N - 1 : c + nbl;
    const long long st = axis == 0 ? (long long)d1 * d2 : (axis == 1 ? (long long)d2 : 1LL);
    const long long base = ((long long)(axis == 0 ? 0 : i) * d1 + (axis == 1 ? 0 : j)) * d2 + (axis == 2 ? 0 : k);
    float s = 0.f;
    for (int t = lo; t <= hi; t++) s += in[base + t * st];
    out[q] = s;
}

// stack[ox + i][oy + j][oz + k] += weight * img[i][j][k]  (img [nx][ny][nz],
// stack [gx][gy][gz]; the window lies inside the stack)
__global__ void stack_kernel(const float *__restrict__ img, float *stack, int nx, int ny, int nz, int gy, int gz,
                             int ox, int oy, int oz, float weight)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q % nz), j = (int)((q / nz) % ny), i = (int)(q / ((long long)nz * ny));
        stack[((long long)(ox + i) * gy + (oy + j)) * gz + (oz + k)] += weight * img[q];
    }
}

__global__ void zeta_kernel(long long n, const float *__restrict__ eps, const float *__restrict__ del,
                            const float *__restrict__ lp, const float *__restrict__ lr,
                            float *__restrict__ zp, float *__restrict__ zr)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float a = 1.f + 2.f * eps[q], s = sqrtf(1.f + 2.f * del[q]);
    const float p = lp[q], r = lr[q];
    zp[q] = a * p + s * r;
    zr[q] = s * p + r;
}

__global__ void ratio_kernel(const float *__restrict__ a, float s, float *out, long long n)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < n) out[q] = s / a[q];
}

__global__ void diff_kernel(const float *a, const float *b, float *out, long long n)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < n) out[q] = a[q] - b[q];
}

// deterministic two-stage sum of squares (double)
__global__ void sumsq_partial(const float *__restrict__ a, long long n, double *part)
{
    __shared__ double sh[NB];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)a[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = NB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// ---- snapshot codec -------------------------------------------------------
__global__ void absmax_partial(const float *__restrict__ a, long long n, float *part)
{
    __shared__ float sh[NB];
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s = fmaxf(s, fabsf(a[i]));
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = NB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// one block: scale = amax / target (1 if amax == 0)
__global__ void absmax_final(const float *part, int np, float target, float *scale)
{
    __shared__ float sh[NB];
    float s = 0.f;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s = fmaxf(s, part[i]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = NB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *scale = sh[0] > 0.f ? sh[0] / target : 1.f;
}

// round-to-nearest-even conversions written from the IEEE formats
__device__ __forceinline__ uint16_t f2bf16(float f)
{
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf162f(uint16_t b) { return __uint_as_float(((uint32_t)b) << 16); }

__global__ void quant_kernel(const float *__restrict__ in, long long n, uint16_t *__restrict__ out,
                             const float *__restrict__ scale, int bf16)
{
    const float inv = 1.f / *scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = in[i] * inv;
        out[i] = bf16 ? f2bf16(v) : __half_as_ushort(__float2half_rn(v));
    }
}
__global__ void dequant_kernel(const uint16_t *__restrict__ in, long long n, const float *__restrict__ scale,
                               int bf16, float *__restrict__ out)
{
    const float s = *scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint16_t b = in[i];
        out[i] = s * (bf16 ? bf162f(b) : __half2float(__ushort_as_half(b)));
    }
}
}  // namespace

// ---------------------------------------------------------------------------
int sp_host_tables(prop_s *P, const float *xyz, int n, const int *trace_of_point, SpHost &T)
{
    const GridDev &g = P->g;
    T = SpHost{};
    T.ridx.assign((size_t)n * 8, 0);
    T.rw.assign((size_t)n * 8, 0.f);
    std::vector<std::tuple<long long, int, float>> ent;
    ent.reserve((size_t)n * 8);
    const int dims[3] = {g.NX, g.NY, g.NZ};
    for (int i = 0; i < n; i++) {
        double s[3], f[3];
        int i0[3];
        for (int a = 0; a < 3; a++) {
            s[a] = (double)xyz[3 * i + a] / (double)g.h + (double)(a == 1 ? g.nby : g.nbl);
            if (!(s[a] >= 0.0) || s[a] > (double)(dims[a] - 1))
                return wp_fail(P, PROP_EINVAL, "sparse point " + std::to_string(i) + " outside the grid");
            i0[a] = (int)std::floor(s[a]);
            f[a] = s[a] - i0[a];
        }
        int c = 0;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int d = 0; d < 2; d++, c++) {
                    const double wt = (a ? f[0] : 1 - f[0]) * (b ? f[1] : 1 - f[1]) * (d ? f[2] : 1 - f[2]);
                    if (wt == 0.0) continue;
                    const long long q = ((long long)(i0[0] + a) * g.NY + (i0[1] + b)) * g.NZ + (i0[2] + d);
                    T.ridx[8 * (size_t)i + c] = q;
                    T.rw[8 * (size_t)i + c] = (float)wt;
                    ent.emplace_back(q, trace_of_point ? trace_of_point[i] : i, (float)wt);
                }
    }
    std::stable_sort(ent.begin(), ent.end(),
                     [](const auto &A, const auto &B) { return std::get<0>(A) < std::get<0>(B); });
    for (size_t e = 0; e < ent.size(); e++) {
        if (e == 0 || std::get<0>(ent[e]) != std::get<0>(ent[e - 1])) {
            T.cells.push_back(std::get<0>(ent[e]));
            T.ptr.push_back((int)e);
        }
        T.trs.push_back(std::get<1>(ent[e]));
        T.ws.push_back(std::get<2>(ent[e]));
    }
    T.ptr.push_back((int)ent.size());
    return PROP_OK;
}

int sp_build(prop_s *P, const float *xyz, int n, const int *trace_of_point, SparseDev *S)
{
    SpHost T;
    WP_TRY(sp_host_tables(P, xyz, n, trace_of_point, T));
    // one block, each table 256-byte aligned
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_ri = T.ridx.size() * sizeof(long long), b_rw = T.rw.size() * sizeof(float),
                 b_c = std::max<size_t>(1, T.cells.size()) * sizeof(long long), b_p = T.ptr.size() * sizeof(int),
                 b_t = std::max<size_t>(1, T.trs.size()) * sizeof(int),
                 b_w = std::max<size_t>(1, T.ws.size()) * sizeof(float);
    const size_t total = up(b_ri) + up(b_rw) + up(b_c) + up(b_p) + up(b_t) + up(b_w);
    sp_free(S);
    WP_TRY(wp_malloc(P, &S->blk, total, "sparse-point tables"));
    unsigned char *q = (unsigned char *)S->blk;
    S->rec_idx = (long long *)q; q += up(b_ri);
    S->rec_w = (float *)q; q += up(b_rw);
    S->cell = (long long *)q; q += up(b_c);
    S->cell_ptr = (int *)q; q += up(b_p);
    S->ent_trace = (int *)q; q += up(b_t);
    S->ent_w = (float *)q;
    S->n = n;
    S->ncell = (int)T.cells.size();
    auto cp = [&](void *dst, const void *src, size_t bytes) -> int {
        if (bytes) WP_CK(P, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, P->stream));
        return PROP_OK;
    };
    WP_TRY(cp(S->rec_idx, T.ridx.data(), b_ri));
    WP_TRY(cp(S->rec_w, T.rw.data(), b_rw));
    WP_TRY(cp(S->cell, T.cells.data(), T.cells.size() * sizeof(long long)));
    WP_TRY(cp(S->cell_ptr, T.ptr.data(), b_p));
    WP_TRY(cp(S->ent_trace, T.trs.data(), T.trs.size() * sizeof(int)));
    WP_TRY(cp(S->ent_w, T.ws.data(), T.ws.size() * sizeof(float)));
    WP_CK(P, cudaStreamSynchronize(P->stream));   // the host tables go out of scope
    return PROP_OK;
}

void sp_free(SparseDev *S)
{
    if (S->blk) cudaFree(S->blk);
    *S = SparseDev{};
}

void sp_record(prop_s *P, const SparseDev *S, const float *f0, const float *f1, const float *f2,
               float scale, float *out_col, const int *tdev)
{
    if (S->n <= 0) return;
    record_kernel<<<nblk(S->n), NB, 0, P->stream>>>(S->n, S->rec_idx, S->rec_w, f0, f1, f2, scale, out_col,
                                                    tdev);
    P->kern_launches++;
}

__global__ void tick_kernel(int *t, int d) { *t += d; }

void k_tick(prop_s *P, int *tdev, int d)
{
    tick_kernel<<<1, 1, 0, P->stream>>>(tdev, d);
    P->kern_launches++;
}

__global__ void set_int_kernel(int *p, int v) { *p = v; }

void k_set_int(prop_s *P, int *p, int v)
{
    set_int_kernel<<<1, 1, 0, P->stream>>>(p, v);
    P->kern_launches++;
}

void sp_inject(prop_s *P, const SparseDev *S, const float *traces, int nt, int t, float scale,
               int mode, float *f0, float *f1, float *f2, const float *grad_u, float *grad, const int *tdev)
{
    if (S->ncell <= 0) return;
    inject_kernel<<<nblk(S->ncell), NB, 0, P->stream>>>(P->g, S->ncell, S->cell, S->cell_ptr,
                                                        S->ent_trace, S->ent_w, traces, nt, t, scale,
                                                        mode, P->m, mode == 3 ? P->eps : P->lam,
                                                        mode == 3 ? P->del : P->mu, f0, f1, f2,
                                                        grad_u, grad, tdev);
    P->kern_launches++;
}

void sp_record_trace_s(prop_s *P, const SparseDev *S, const float *f0, const float *f1,
                       const float *f2, float scale, float *out_col)
{
    if (S->n <= 0) return;
    record_s_kernel<<<nblk(S->n), NB, 0, P->stream>>>(P->g, S->n, S->rec_idx, S->rec_w, f0, f1, f2, P->lam,
                                                      P->mu, f2 ? 3.f : 2.f, scale, out_col);
    P->kern_launches++;
}

void sp_transpose(prop_s *P, const float *in_tn, float *out_nt, int n, int nt)
{
    dim3 blk(32, 8), grd((n + 31) / 32, (nt + 31) / 32);
    transpose_kernel<<<grd, blk, 0, P->stream>>>(in_tn, out_nt, n, nt);
    P->kern_launches++;
}

void k_extend(prop_s *P, const float *phys, float *comp, float scale, int mode)
{
    extend_kernel<<<nblk(P->g.N), NB, 0, P->stream>>>(P->g, phys, comp, scale, mode);
}

void k_lame(prop_s *P)
{
    lame_kernel<<<nblk(P->g.N), NB, 0, P->stream>>>(P->g.N, P->bu, P->lam, P->mu);
}

void k_normals(prop_s *P)
{
    normals_kernel<<<nblk(P->g.N), NB, 0, P->stream>>>(P->g.N, P->th, P->ph, P->nrm[0], P->nrm[1]);
}

void k_fold(prop_s *P, const float *comp, float *phys, float *s1, float *s2)
{
    const GridDev &g = P->g;
    const long long n1 = (long long)g.NX * g.NY * g.pz, n2 = (long long)g.NX * g.py * g.pz,
                    n3 = (long long)g.px * g.py * g.pz;
    fold_axis_kernel<<<nblk(n1), NB, 0, P->stream>>>(comp, s1, g.NX, g.NY, g.NZ, 2, g.pz, g.nbl);
    fold_axis_kernel<<<nblk(n2), NB, 0, P->stream>>>(s1, s2, g.NX, g.NY, g.pz, 1, g.py, g.nby);
    fold_axis_kernel<<<nblk(n3), NB, 0, P->stream>>>(s2, phys, g.NX, g.py, g.pz, 0, g.px, g.nbl);
    P->kern_launches += 3;
}

void k_ratio(prop_s *P, const float *a, float s, float *out, long long n)
{
    ratio_kernel<<<nblk(n), NB, 0, P->stream>>>(a, s, out, n);
    P->kern_launches += 1;
}

void k_stack(prop_s *P, const float *img, float *stack, const int *gdims, const int *off, float weight)
{
    const long long n = (long long)P->g.px * P->g.py * P->g.pz;
    stack_kernel<<<nblk(n), NB, 0, P->stream>>>(img, stack, P->g.px, P->g.py, P->g.pz, gdims[1], gdims[2], off[0],
                                                off[1], off[2], weight);
    P->kern_launches += 1;
}

void k_tti_zeta(prop_s *P, const float *lp, const float *lr, float *zp, float *zr)
{
    zeta_kernel<<<nblk(P->g.N), NB, 0, P->stream>>>(P->g.N, P->eps, P->del, lp, lr, zp, zr);
    P->kern_launches += 1;
}

void k_axpy_sq(prop_s *P, const float *a, const float *b, float *out, long long n)
{
    diff_kernel<<<nblk(n), NB, 0, P->stream>>>(a, b, out, n);
    P->kern_launches++;
}

int k_sumsq(prop_s *P, const float *a, long long n, double *out)
{
    const int nb = 1024;
    *out = 0.0;
    if (!P->sumsq) WP_TRY(wp_malloc(P, (void **)&P->sumsq, sizeof(double) * nb, "misfit partial sums"));
    sumsq_partial<<<nb, NB, 0, P->stream>>>(a, n, P->sumsq);
    P->kern_launches++;
    WP_CK(P, cudaGetLastError());
    std::vector<double> h(nb);
    WP_CK(P, cudaMemcpyAsync(h.data(), P->sumsq, sizeof(double) * nb, cudaMemcpyDeviceToHost, P->stream));
    WP_CK(P, cudaStreamSynchronize(P->stream));
    double s = 0.0;
    for (double v : h) s += v;
    *out = s;
    return PROP_OK;
}

void k_snap_encode(prop_s *P, const float *in, long long n, uint16_t *out, float *scale_dev,
                   int bf16, float *scratch)
{
    const int nb = 1024;   // scratch holds nb partial maxima
    absmax_partial<<<nb, NB, 0, P->stream>>>(in, n, scratch);
    absmax_final<<<1, NB, 0, P->stream>>>(scratch, nb, bf16 ? 1.f : 32768.f, scale_dev);
    quant_kernel<<<std::min(nblk(n), 152 * 16), NB, 0, P->stream>>>(in, n, out, scale_dev, bf16);
    P->kern_launches += 3;
}

void k_snap_decode(prop_s *P, const uint16_t *in, long long n, const float *scale_dev, int bf16,
                   float *out)
{
    dequant_kernel<<<std::min(nblk(n), 152 * 16), NB, 0, P->stream>>>(in, n, scale_dev, bf16, out);
    P->kern_launches++;
}
