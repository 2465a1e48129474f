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
// stays reserved until the process exits.  Each call looks up the array's
// device address (cudaGetSymbolAddress with the device current) unless the
// stream is being captured, in which case the address found by the last
// uncaptured call on that device is used: make one call on a device before
// any stream capture starts there.  A device reset (cudaDeviceReset) unloads
// the module; the next uncaptured call finds the new address.  All calls
// share the array and it keeps the contents of the last call: everything
// that must start at zero is cleared on every call, and calls that overlap on
// the GPU (concurrent streams, or threads calling at once) race on the same
// memory.  A call that fails after queuing work waits for that work before
// it returns, so a failed call never leaves kernels running on the array.
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
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    WP_CK(P, cudaStreamIsCapturing(P->stream, &cap));
    std::lock_guard<std::mutex> lk(g_mtx);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return wp_cuda(P, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_addr[dev] = p;
    } else if (!g_addr[dev]) {
        return wp_fail(P, PROP_EINVAL, "first prop_forward_noalloc call on a device must not be captured");
    }
    *out = (unsigned char *)g_addr[dev];
    return PROP_OK;
}

// waits for the queued work of a failed call (its status is not reported)
struct SyncOnExit {
    cudaStream_t s;
    bool armed = false;
    ~SyncOnExit()
    {
        if (armed) {
            cudaStreamSynchronize(s);
            cudaGetLastError();
        }
    }
};

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

// carve device space for one table set and (if placed) copy it in
int place_tables(prop_s *P, Carver &C, const SpHost &T, int n, SparseDev &S)
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
    // sizes checked before any product can overflow: each computational axis,
    // then the point count (< 2^32, 32-bit offsets in the kernels), then one
    // field's bytes and every field's bytes against the static array
    const long long ax[3] = {(long long)d->nx + 2LL * d->nbl, (long long)d->ny + 2LL * d->nbl,
                             (long long)d->nz + 2LL * d->nbl};
    for (long long a : ax)
        if (a > (long long)WP_NOALLOC_BYTES)
            return wp_fail(P, PROP_EINVAL, "grid axis too long for prop_forward_noalloc");
    const unsigned long long nxy = (unsigned long long)ax[0] * (unsigned long long)ax[1];
    if (nxy >= (1ull << 32) || nxy * (unsigned long long)ax[2] >= (1ull << 32))
        return wp_fail(P, PROP_EINVAL, "computational grid above 2^32 - 1 points");
    const unsigned long long nfield = (tti ? 7 + 4 + 6 : 3 + 9);
    const unsigned long long fbytes = nxy * (unsigned long long)ax[2] * sizeof(float);
    if (fbytes > WP_NOALLOC_BYTES || fbytes * nfield > WP_NOALLOC_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "problem needs more than %.1f MiB of device scratch; prop_forward_noalloc holds %u MiB",
                 fbytes * (double)nfield / 1048576.0, WP_NOALLOC_BYTES >> 20);
        return wp_fail(P, PROP_EINVAL, buf);
    }
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
    SpHost TS, TR;
    if (int rc = sp_host_tables(P, hs.data(), nsrc, nullptr, TS)) return rc;
    if (int rc = sp_host_tables(P, hr.data(), nrec, nullptr, TR)) return rc;
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
    SyncOnExit guard{P->stream};
    guard.armed = true;               // from here on work may be queued
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
    guard.armed = false;
    WP_CK(P, cudaGetLastError());
    int f = 0;
    WP_CK(P, cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost));
    return wp_flag_status(P, f);
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
