// prop_forward_noalloc: forward modelling that never allocates device memory.
//
// Some callers cannot call cudaMalloc: a host application whose own
// allocator has reserved the GPU's memory up front and hands out blocks
// itself, or a latency-bound service that forbids device allocation after
// start-up because cudaMalloc/cudaFree can synchronize the device and take
// unbounded time.  For them this entry point does the same work as
// prop_create + prop_forward + prop_destroy with every device buffer it needs
// (computational-grid model, wavefield state, intermediate fields, staging
// of the wavelet and traces, source/receiver tables) carved out of one
// file-scope static __device__ array of WP_NOALLOC_BYTES.
//
// The array belongs to this library's code on each GPU: it is reserved on a
// device when that device loads the module holding it (with CUDA's default
// lazy module loading, at the first call of this entry point there) and it
// stays reserved until the process exits.  The first call on a device looks
// up the array's device address (cudaGetSymbolAddress with that device
// current) and caches it; that first call should come before any stream
// capture is started on that device.  All calls share the array and it keeps
// the contents of the last call: everything that must start at zero is
// cleared on every call, and calls that overlap on the GPU (concurrent
// streams, or threads calling at once) race on the same memory.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <tuple>

#define WP_NOALLOC_BYTES (48u << 20)   // 48 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[WP_NOALLOC_BYTES];

namespace {

std::mutex g_mtx;
void *g_addr[256] = {};

int scratch_address(prop_s *P, unsigned char **out)
{
    int dev = 0;
    WP_CK(P, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return wp_fail(P, PROP_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mtx);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return wp_cuda(P, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return PROP_OK;
}

// sequential sub-allocation of the static array (base == nullptr: sizing pass)
struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <class T> T *take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

// trilinear tables (same layout as the library's own sparse tables)
struct HostTables {
    std::vector<long long> ridx, cells;
    std::vector<float> rw, ws;
    std::vector<int> ptr, trs;
};

int host_tables(prop_s *P, const float *xyz, int n, HostTables &T)
{
    const GridDev &g = P->g;
    T.ridx.assign((size_t)n * 8, 0);
    T.rw.assign((size_t)n * 8, 0.f);
    std::vector<std::tuple<long long, int, float>> ent;
    const int dims[3] = {g.NX, g.NY, g.NZ};
    for (int i = 0; i < n; i++) {
        double s[3], f[3];
        int i0[3];
        for (int a = 0; a < 3; a++) {
            s[a] = (double)xyz[3 * i + a] / (double)g.h + (double)g.nbl;
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
                    ent.emplace_back(q, i, (float)wt);
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

// carve device space for one table set and (if placed) copy it in
int place_tables(prop_s *P, Carver &C, const HostTables &T, int n, SparseDev &S)
{
    S.n = n;
    S.ncell = (int)T.cells.size();
    S.rec_idx = C.take<long long>(T.ridx.size());
    S.rec_w = C.take<float>(T.rw.size());
    S.cell = C.take<long long>(std::max<size_t>(1, T.cells.size()));
    S.cell_ptr = C.take<int>(T.ptr.size());
    S.ent_trace = C.take<int>(std::max<size_t>(1, T.trs.size()));
    S.ent_w = C.take<float>(std::max<size_t>(1, T.ws.size()));
    if (!C.base) return PROP_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes) -> int {
        if (bytes) WP_CK(P, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, P->stream));
        return PROP_OK;
    };
    if (int rc = cp(S.rec_idx, T.ridx.data(), T.ridx.size() * sizeof(long long))) return rc;
    if (int rc = cp(S.rec_w, T.rw.data(), T.rw.size() * sizeof(float))) return rc;
    if (int rc = cp(S.cell, T.cells.data(), T.cells.size() * sizeof(long long))) return rc;
    if (int rc = cp(S.cell_ptr, T.ptr.data(), T.ptr.size() * sizeof(int))) return rc;
    if (int rc = cp(S.ent_trace, T.trs.data(), T.trs.size() * sizeof(int))) return rc;
    return cp(S.ent_w, T.ws.data(), T.ws.size() * sizeof(float));
}

int run(prop_s *P, const prop_desc *d, const float *const *model, const float *wavelet,
        const float *src, int nsrc, const float *rec, int nrec, float *traces)
{
    // ---- validation (the rules of prop_create / prop_forward) -----------
    const int so = d->space_order;
    if (d->kind != PROP_TTI && d->kind != PROP_ELASTIC) return wp_fail(P, PROP_EINVAL, "kind must be PROP_TTI or PROP_ELASTIC");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nbl < 0) return wp_fail(P, PROP_EINVAL, "bad grid sizes");
    if (d->tti_operator != 0) return wp_fail(P, PROP_EINVAL, "prop_forward_noalloc needs tti_operator = 0");
    if (!(d->h > 0.f) || !std::isfinite(d->h)) return wp_fail(P, PROP_EINVAL, "h must be > 0");
    if (so != 4 && so != 8 && so != 12 && so != 16) return wp_fail(P, PROP_EINVAL, "space_order must be 4, 8, 12 or 16");
    if (d->nt < 2) return wp_fail(P, PROP_EINVAL, "nt must be >= 2");
    if (nsrc < 1 || nrec < 1) return wp_fail(P, PROP_EINVAL, "nsrc and nrec must be >= 1");
    if (!model || !wavelet || !src || !rec || !traces) return wp_fail(P, PROP_EINVAL, "NULL argument");
    const bool tti = d->kind == PROP_TTI;
    const int nf = tti ? 5 : 3;
    for (int i = 0; i < nf; i++)
        if (!model[i]) return wp_fail(P, PROP_EINVAL, "model array is NULL");
    P->d = *d;
    P->M = so / 2;
    GridDev &g = P->g;
    g.nbl = d->nbl; g.nby = d->nbl; g.px = d->nx; g.py = d->ny; g.pz = d->nz;
    g.NX = d->nx + 2 * d->nbl; g.NY = d->ny + 2 * d->nbl; g.NZ = d->nz + 2 * d->nbl;
    g.N = (long long)g.NX * g.NY * g.NZ;
    g.h = d->h; g.ih = 1.f / d->h; g.cer = 0.015f;
    if (!fd_weights(P->M, P->w.c, P->w.b)) return wp_fail(P, PROP_EINVAL, "FD weights");
    const size_t np = (size_t)d->nx * d->ny * d->nz, N = (size_t)g.N;
    const int nt = d->nt;

    // ---- scratch layout (sizing pass first) ------------------------------
    std::vector<float> hs((size_t)nsrc * 3), hr((size_t)nrec * 3);
    WP_CK(P, cudaMemcpy(hs.data(), src, hs.size() * 4, cudaMemcpyDefault));
    WP_CK(P, cudaMemcpy(hr.data(), rec, hr.size() * 4, cudaMemcpyDefault));
    HostTables TS, TR;
    if (int rc = host_tables(P, hs.data(), nsrc, TS)) return rc;
    if (int rc = host_tables(P, hr.data(), nrec, TR)) return rc;
    SparseDev S, R;
    float *phys, *wav, *stage, *out, *tabd, *fields[20] = {};
    int *flag;
    const size_t ntab = (size_t)(g.NX + g.NY + g.NZ) * (tti ? 1 : 2);
    const int nmodel = tti ? 7 : 3, nstate = tti ? 4 : 9, ntmp = tti ? 6 : 0;
    auto layout = [&](Carver &C) -> int {
        for (int i = 0; i < nmodel + nstate + ntmp; i++) fields[i] = C.take<float>(N);
        phys = C.take<float>(np);
        wav = C.take<float>((size_t)nsrc * nt);
        stage = C.take<float>((size_t)nrec * nt);
        out = C.take<float>((size_t)nrec * nt);
        flag = C.take<int>(1);
        tabd = C.take<float>(ntab);
        if (int rc = place_tables(P, C, TS, nsrc, S)) return rc;
        return place_tables(P, C, TR, nrec, R);
    };
    Carver sizing{nullptr};
    layout(sizing);
    if (sizing.off > WP_NOALLOC_BYTES) {
        char buf[240];
        snprintf(buf, sizeof buf,
                 "problem needs %.1f MiB of device scratch; prop_forward_noalloc holds %u MiB "
                 "(use prop_create/prop_forward for larger problems)",
                 sizing.off / 1048576.0, WP_NOALLOC_BYTES >> 20);
        return wp_fail(P, PROP_EINVAL, buf);
    }

    // ---- model on the host: validation, dt, CFL, damping -------------------
    std::vector<std::vector<float>> hm(nf);
    for (int i = 0; i < nf; i++) {
        hm[i].resize(np);
        WP_CK(P, cudaMemcpy(hm[i].data(), model[i], np * sizeof(float), cudaMemcpyDefault));
    }
    double vmax = 0.0;
    for (size_t q = 0; q < np; q++) {
        const float vp = hm[0][q];
        if (!(vp > 0.f) || !std::isfinite(vp)) return wp_fail(P, PROP_EINVAL, "vp must be finite and > 0");
        if (tti) {
            const float e = hm[1][q], dl = hm[2][q];
            if (!std::isfinite(e) || !std::isfinite(dl) || !std::isfinite(hm[3][q]) || !std::isfinite(hm[4][q]))
                return wp_fail(P, PROP_EINVAL, "non-finite TTI parameter");
            if (e < dl) return wp_fail(P, PROP_EINVAL, "epsilon < delta somewhere (TTI stability needs eps >= delta)");
            if (1.0 + 2.0 * dl <= 0.0) return wp_fail(P, PROP_EINVAL, "1 + 2 delta must be > 0");
            vmax = std::max(vmax, 1000.0 * vp * sqrt(1.0 + 2.0 * e));
        } else {
            const float vs = hm[1][q], rho = hm[2][q];
            if (!(vs >= 0.f) || !std::isfinite(vs)) return wp_fail(P, PROP_EINVAL, "vs must be finite and >= 0");
            if (!(rho > 0.f) || !std::isfinite(rho)) return wp_fail(P, PROP_EINVAL, "rho must be finite and > 0");
            if ((double)vp * vp < 2.0 * (double)vs * vs) return wp_fail(P, PROP_EINVAL, "lambda < 0 (vp^2 < 2 vs^2)");
            vmax = std::max(vmax, 1000.0 * vp);
        }
    }
    const double dt = d->dt > 0.f ? (double)d->dt : 0.4 * d->h / vmax;
    g.dt = (float)dt;
    P->d.dt = g.dt;
    const double lim = 2.0 / (sqrt(3.0) * symbol_max(tti ? P->w.c : P->w.b, P->M, !tti));
    if (vmax * dt / d->h > lim) return wp_fail(P, PROP_EUNSTABLE, "dt above the CFL stability bound");
    if (d->nbl > 0) {
        const double L = d->nbl * (double)d->h;
        const double vd = d->vdamp > 0.f ? (double)d->vdamp : vmax;
        g.sig0 = (float)(3.0 * vd / (2.0 * L) * log(1000.0));
    }

    // ---- place everything in the static array -----------------------------
    unsigned char *base = nullptr;
    if (int rc = scratch_address(P, &base)) return rc;
    Carver C{base};
    if (int rc = layout(C)) return rc;
    int k = 0;
    if (tti) {
        P->m = fields[k++]; P->eps = fields[k++]; P->del = fields[k++]; P->th = fields[k++]; P->ph = fields[k++];
        P->nrm[0] = fields[k++]; P->nrm[1] = fields[k++];
    } else {
        P->bu = fields[k++]; P->lam = fields[k++]; P->mu = fields[k++];
    }
    for (int i = 0; i < nstate; i++) P->st[i] = fields[k++];
    for (int i = 0; i < ntmp; i++) P->tmp[i] = fields[k++];
    P->flag = flag;
    const std::vector<float> tabh = layer_tables(g, d->kind);     // after sig0 is known
    WP_CK(P, cudaMemcpyAsync(tabd, tabh.data(), tabh.size() * sizeof(float), cudaMemcpyHostToDevice,
                             P->stream));
    g.tab = tabd;
    {
        int dev = 0, sms = 152;
        WP_CK(P, cudaGetDevice(&dev));
        WP_CK(P, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        P->xchunk = stencil_xchunk(g, sms);
    }
    float *mdst[5] = {tti ? P->m : P->bu, tti ? P->eps : P->lam, tti ? P->del : P->mu, P->th, P->ph};
    for (int i = 0; i < nf; i++) {
        WP_CK(P, cudaMemcpyAsync(phys, hm[i].data(), np * sizeof(float), cudaMemcpyHostToDevice, P->stream));
        k_extend(P, phys, mdst[i], (tti && i == 0) ? 1000.f : 1.f, (tti && i == 0) ? 1 : 0);
    }
    if (!tti) k_lame(P);
    else k_normals(P);
    WP_CK(P, cudaMemcpyAsync(wav, wavelet, (size_t)nsrc * nt * sizeof(float), cudaMemcpyDefault, P->stream));
    for (int i = 0; i < nstate; i++) WP_CK(P, cudaMemsetAsync(P->st[i], 0, N * sizeof(float), P->stream));
    WP_CK(P, cudaMemsetAsync(flag, 0, sizeof(int), P->stream));

    // ---- time loop (record d^n from u^n, advance, inject q^n) ---------------
    float *s[9];
    for (int i = 0; i < nstate; i++) s[i] = P->st[i];
    for (int n = 0; n < nt; n++) {
        if (tti) sp_record(P, &R, s[0], nullptr, nullptr, 1.f, stage + (size_t)n * nrec);
        else sp_record(P, &R, s[3], s[4], s[5], 1.f, stage + (size_t)n * nrec);
        if (tti) {
            if (int rc = tti_launch_step(P, s, false, nullptr, nullptr, nullptr)) return rc;
            std::swap(s[0], s[2]);
            std::swap(s[1], s[3]);
            sp_inject(P, &S, wav, nt, n, g.dt * g.dt, 1, s[0], s[1], nullptr, nullptr, nullptr);
        } else {
            if (int rc = el_launch_step(P, s, false)) return rc;
            sp_inject(P, &S, wav, nt, n, g.dt, 0, s[3], s[4], s[5], nullptr, nullptr);
        }
    }
    sp_transpose(P, stage, out, nrec, nt);
    WP_CK(P, cudaMemcpyAsync(traces, out, (size_t)nrec * nt * sizeof(float), cudaMemcpyDefault, P->stream));
    WP_CK(P, cudaStreamSynchronize(P->stream));
    WP_CK(P, cudaGetLastError());
    if (d->check_nan) {
        int f = 0;
        WP_CK(P, cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (f) return wp_fail(P, PROP_EUNSTABLE, "NaN or Inf in the wavefield");
    }
    return PROP_OK;
}

}  // namespace

extern "C" int prop_forward_noalloc(const prop_desc *desc, const float *const *model,
                                    const float *wavelet, const float *src_xyz, int nsrc,
                                    const float *rec_xyz, int nrec, float *traces, void *cuda_stream)
{
    if (!desc) return wp_fail(nullptr, PROP_EINVAL, "desc is NULL");
    prop_s P;                       // host bookkeeping only; device pointers point into the array
    P.stream = (cudaStream_t)cuda_stream;
    int rc = run(&P, desc, model, wavelet, src_xyz, nsrc, rec_xyz, nrec, traces);
    if (rc) wp_fail(nullptr, rc, P.err);   // message for prop_last_error(NULL)
    return rc;
}
