// Host runtime and C ABI of waveprop (declared in include/waveprop.h).
//
// Time loops follow the order of the Sec. II-A listing: per step n record
// d^n from u^n, advance, inject q^n into the new level.  Adjoint loops run
// the transposed steps backwards.  Gradients use the adjoint-state method
// (Sec. III) with forward wavefields either kept in full or recomputed from
// checkpoints (FP32, or BF16/FP16 with one scale per field).  Source-free
// state steps (prop_step) replay pairs of steps from a CUDA graph captured
// once per handle, direction and state buffers.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <memory>
#include <thread>
#include <functional>

static thread_local std::string tl_err;

int wp_fail(prop_s *P, int code, const std::string &msg)
{
    tl_err = msg;
    if (P) {
        P->err = msg;
        if (code == PROP_ECUDA || code == PROP_ETIMEOUT) P->broken = true;
    }
    return code;
}

int wp_cuda(prop_s *P, cudaError_t e, const char *what)
{
    std::string m = std::string("CUDA error '") + cudaGetErrorString(e) + "' in " + what;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return wp_fail(P, PROP_ENOMEM, m);
    }
    return wp_fail(P, PROP_ECUDA, m);
}

// All device allocations of the library go through here (prop_forward_noalloc
// makes none).  WAVEPROP_FAULT=alloc makes every allocation fail (host-side
// fault injection for tests).
int wp_dev_alloc(void **p, size_t bytes, const char *what, std::string *msg)
{
    *p = nullptr;
    const char *f = getenv("WAVEPROP_FAULT");
    if (f && !strcmp(f, "alloc")) {
        if (msg) *msg = std::string("injected allocation failure: ") + what;
        return PROP_ENOMEM;
    }
    const cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) return PROP_OK;
    *p = nullptr;
    char buf[200];
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        snprintf(buf, sizeof buf, "cannot allocate %.3f GB for %s", bytes / 1e9, what);
        if (msg) *msg = buf;
        return PROP_ENOMEM;
    }
    snprintf(buf, sizeof buf, "CUDA error '%s' allocating %.3f GB for %s", cudaGetErrorString(e), bytes / 1e9, what);
    if (msg) *msg = buf;
    return PROP_ECUDA;
}
int wp_malloc(prop_s *P, void **p, size_t bytes, const char *what)
{
    std::string m;
    const int rc = wp_dev_alloc(p, bytes, what, &m);
    return rc ? wp_fail(P, rc, m) : PROP_OK;
}
#define WP_MALLOC(P, ptr, bytes, what)                                            \
    do {                                                                          \
        int _r = wp_malloc((P), (void **)&(ptr), (bytes), (what));                \
        if (_r) return _r;                                                        \
    } while (0)

// ---------------------------------------------------------------------------
// FD weights: solve the moment conditions in double precision
//   centred:   sum_k c_k 2 k^(2j+1)       = [j == 0],  j = 0..M-1
//   staggered: sum_k b_k 2 (k-1/2)^(2j+1) = [j == 0]
// ---------------------------------------------------------------------------
static bool solve_dense(int n, std::vector<double> &A, std::vector<double> &b)
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; k++) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; r++) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return true;
}

bool fd_weights(int M, float *c, float *bst)
{
    for (int stag = 0; stag < 2; stag++) {
        std::vector<double> A(M * M), b(M, 0.0);
        for (int j = 0; j < M; j++)
            for (int k = 1; k <= M; k++) {
                double off = stag ? k - 0.5 : (double)k;
                A[j * M + (k - 1)] = 2.0 * pow(off, 2 * j + 1);
            }
        b[0] = 1.0;
        if (!solve_dense(M, A, b)) return false;
        for (int k = 0; k < M; k++) (stag ? bst : c)[k] = (float)b[k];
    }
    for (int k = M; k < WP_MAXM; k++) c[k] = bst[k] = 0.f;
    return true;
}

// centred second derivative, closed form:
//   d2_k = 2 (-1)^(k+1) (M!)^2 / (k^2 (M-k)! (M+k)!),  d2_0 = -2 sum_k d2_k
static void d2_weights(int M, float *d2)
{
    double s = 0.0;
    for (int k = 1; k <= M; k++) {
        double r = 1.0;                       // (M!)^2 / ((M-k)! (M+k)!)
        for (int j = 1; j <= k; j++) r *= (double)(M - k + j) / (double)(M + j);
        const double v = (k % 2 ? 2.0 : -2.0) * r / ((double)k * k);
        d2[k] = (float)v;
        s += v;
    }
    d2[0] = (float)(-2.0 * s);
    for (int k = M + 1; k <= WP_MAXM; k++) d2[k] = 0.f;
}

// max over kappa of |d2_0 + 2 sum_k d2_k cos(k kappa)| (1D symbol of h^2 D2)
static double symbol2_max(const float *d2, int M)
{
    double mx = 0.0;
    for (int i = 0; i <= 4096; i++) {
        double kap = M_PI * i / 4096.0, s = d2[0];
        for (int k = 1; k <= M; k++) s += 2.0 * d2[k] * cos(k * kap);
        mx = std::max(mx, fabs(s));
    }
    return mx;
}

// max over kappa of |sum_k 2 w_k sin(s_k kappa)| (s_k = k or k - 1/2)
double symbol_max(const float *w, int M, bool stag)
{
    double mx = 0.0;
    for (int i = 0; i <= 4096; i++) {
        double kap = M_PI * i / 4096.0, s = 0.0;
        for (int k = 1; k <= M; k++) s += 2.0 * w[k - 1] * sin((stag ? k - 0.5 : (double)k) * kap);
        mx = std::max(mx, fabs(s));
    }
    return mx;
}

// Absorbing-layer factors are separable per axis: the TTI damping rate is a
// sum sig0 (d/L)^2 over axes, the elastic Cerjan taper a product
// exp(-(0.015 d)^2) over axes (d = depth into the layer in cells, at the
// node or at the half point of a staggered component).
std::vector<float> layer_tables(const GridDev &g, int kind)
{
    auto depth = [&](double s, int a) {
        const int nb = a == 1 ? g.nby : g.nbl, n = a == 0 ? g.px : (a == 1 ? g.py : g.pz);
        const double lo = nb, hi = nb + n - 1;
        return s < lo ? lo - s : (s > hi ? s - hi : 0.0);
    };
    const int NN[3] = {g.NX, g.NY, g.NZ};
    std::vector<float> t;
    for (int a = 0; a < 3; a++)
        for (int i = 0; i < NN[a]; i++) {
            if (kind == PROP_TTI || kind == PROP_ACOUSTIC) {   // damping rate
                const double d = g.nbl > 0 ? depth(i, a) / g.nbl : 0.0;
                t.push_back((float)((double)g.sig0 * d * d));
            } else {
                for (int hf = 0; hf < 2; hf++) {
                    const double d = g.nbl > 0 ? (double)g.cer * depth(i + 0.5 * hf, a) : 0.0;
                    t.push_back((float)exp(-d * d));
                }
            }
        }
    return t;
}

// ---------------------------------------------------------------------------
// pointers: host or device
// ---------------------------------------------------------------------------
static bool is_dev(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DevBuf {   // RAII device buffer owned by one call
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

// device view of a caller buffer of n floats (copied in if host)
static int dev_in(prop_s *P, const float *src, size_t n, DevBuf &tmp, const float **out)
{
    if (is_dev(src)) {
        *out = src;
        return PROP_OK;
    }
    WP_TRY(wp_malloc(P, &tmp.p, n * sizeof(float), "input staging"));
    WP_CK(P, cudaMemcpyAsync(tmp.p, src, n * sizeof(float), cudaMemcpyHostToDevice, P->stream));
    *out = (const float *)tmp.p;
    return PROP_OK;
}
static int copy_out(prop_s *P, float *dst, const float *src_dev, size_t n)
{
    WP_CK(P, cudaMemcpyAsync(dst, src_dev, n * sizeof(float), cudaMemcpyDefault, P->stream));
    return PROP_OK;
}

// state fields: TTI (p, r) at two levels, acoustic u at two levels, elastic 9,
// 2D elastic 5
static int nfields(const prop_s *P)
{
    switch (P->d.kind) {
    case PROP_TTI: return 4;
    case PROP_ACOUSTIC: return 2;
    case PROP_ELASTIC2D: return 5;
    default: return 9;
    }
}

// ---------------------------------------------------------------------------
// profiling
// ---------------------------------------------------------------------------
void prof_begin(prop_s *P, int id)
{
    if (!P->prof) return;
    if ((size_t)P->prof_used * 2 + 2 > P->prof_ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        P->prof_ev.push_back(a);
        P->prof_ev.push_back(b);
        P->prof_id.push_back(id);
    }
    P->prof_id[P->prof_used] = id;
    cudaEventRecord(P->prof_ev[2 * P->prof_used], P->stream);
}
void prof_end(prop_s *P, int id)
{
    (void)id;
    if (!P->prof) return;
    cudaEventRecord(P->prof_ev[2 * P->prof_used + 1], P->stream);
    P->prof_used++;
}
static void prof_collect(prop_s *P)
{
    if (!P->prof || !P->prof_used) return;
    cudaStreamSynchronize(P->stream);
    for (int i = 0; i < P->prof_used; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P->prof_ev[2 * i], P->prof_ev[2 * i + 1]) == cudaSuccess) {
            P->prof_ms[P->prof_id[i]] += ms;
            P->prof_n[P->prof_id[i]] += 1;
        }
    }
    P->prof_used = 0;
}

// collect events every so often so the pool stays small
static void prof_maybe_collect(prop_s *P)
{
    if (P->prof && P->prof_used >= 256) prof_collect(P);
}

// ---------------------------------------------------------------------------
// creation
// ---------------------------------------------------------------------------
static int ensure_tmp(prop_s *P, int count)
{
    for (int i = 0; i < count; i++)
        if (!P->tmp[i]) WP_MALLOC(P, P->tmp[i], sizeof(float) * P->g.N, "scratch fields");
    return PROP_OK;
}
// state and scratch arrays of a call (prop_trim releases them between calls)
static int ensure_work(prop_s *P)
{
    for (int i = 0; i < nfields(P); i++)
        if (!P->st[i]) {
            WP_MALLOC(P, P->st[i], sizeof(float) * P->g.N, "state");
            WP_CK(P, cudaMemsetAsync(P->st[i], 0, sizeof(float) * P->g.N, P->stream));
        }
    if (P->d.kind == PROP_TTI) return ensure_tmp(P, P->d.tti_operator == 1 ? 14 : 8);
    return PROP_OK;
}
static int ensure_ast(prop_s *P)
{
    for (int i = 0; i < nfields(P); i++)
        if (!P->ast[i]) WP_MALLOC(P, P->ast[i], sizeof(float) * P->g.N, "adjoint state");
    return PROP_OK;
}

static void free_snaps(prop_s *P)
{
    cudaFree(P->tail); P->tail = nullptr; P->tail_bytes = 0; P->tail_T = 0;
    cudaFree(P->snap); P->snap = nullptr; P->snap_bytes = 0;
    cudaFree(P->snap16); P->snap16 = nullptr; P->snap16_bytes = 0;
    cudaFree(P->snap_scale); P->snap_scale = nullptr;
    cudaFree(P->seg); P->seg = nullptr; P->seg_bytes = 0;
    P->saved = false;
    P->tmaps.clear();        // descriptors may name the freed buffers
}

static void free_all(prop_s *P)
{
    float *arrs[] = {P->m, P->eps, P->del, P->th, P->ph, P->nrm[0], P->nrm[1], P->bu, P->lam, P->mu, P->acw};
    for (float *a : arrs) cudaFree(a);
    for (auto &a : P->st) cudaFree(a);
    for (auto &a : P->ast) cudaFree(a);
    for (auto &a : P->tmp) cudaFree(a);
    cudaFree(P->flag);
    cudaFree(P->sumsq);
    cudaFree(P->tab);
    free_snaps(P);
    for (auto e : P->prof_ev) cudaEventDestroy(e);
    if (P->step_graph) cudaGraphExecDestroy(P->step_graph);
    if (P->graph_stream) cudaStreamDestroy(P->graph_stream);
}

static int step_state(prop_s *P, float **s, bool adjoint);
static int zero_fields(prop_s *P, float *const *f, int n);

// ---------------------------------------------------------------------------
// autotuner: tile shape of the stencil passes, i.e. the tile height (rows of
// y per CTA: 8, 16 or 32, each a separately compiled set of TMA passes;
// elastic and centred TTI) and the x-extent (planes per CTA).  The height
// trades the y halo each plane re-fetches (2M rows per tile) against the
// number of CTAs and their size; the x-extent sets the number of CTAs
// (waves on the SMs) against the queue warm-up cost per chunk.  Candidates
// are timed on a few forward steps of the zero state; the choice is cached
// per (kind, space order, grid, TMA path) for the process and, if
// WAVEPROP_AUTOTUNE_CACHE names a file, across processes (lines "key xc ty").
// WAVEPROP_AUTOTUNE=0 keeps the occupancy heuristic at 16 rows;
// WAVEPROP_TILE_Y=8|16|32 fixes the height and tunes only the x-extent.
// Results do not depend on the choice (a point's arithmetic is the same in
// every tile).
// ---------------------------------------------------------------------------
#include <map>
#include <mutex>
#include <sstream>
#include <fstream>

static std::mutex g_tune_mtx;
static std::map<std::string, std::pair<int, int>> g_tune;
static bool g_tune_loaded = false;

static std::string tune_key(const prop_s *P, int forced_ty)
{
    std::ostringstream k;
    k << P->d.kind << ':' << P->M << ':' << P->g.NX << 'x' << P->g.NY << 'x' << P->g.NZ << ':'
      << (tma_usable(P) ? "tma" : "pipe") << ":h" << forced_ty;
    return k.str();
}

// WAVEPROP_TILE_Y: a fixed tile height, or 0 (tuned)
static int forced_tile_y()
{
    const char *v = getenv("WAVEPROP_TILE_Y");
    if (!v) return 0;
    const int t = atoi(v);
    return t == 8 || t == 16 || t == 32 ? t : 0;
}

static int autotune_tiles(prop_s *P)
{
    const char *on = getenv("WAVEPROP_AUTOTUNE");
    const int fty = forced_tile_y();
    const bool tma = tma_usable(P);
    if (fty && tma && tile_height_fits(P, fty)) P->tile_y = fty;
    // the 2D and staggered-pair passes have no x chunks
    if ((on && !strcmp(on, "0")) || P->d.kind == PROP_ELASTIC2D || P->d.tti_operator == 1) return PROP_OK;
    const char *path = getenv("WAVEPROP_AUTOTUNE_CACHE");
    const std::string key = tune_key(P, fty);
    {
        std::lock_guard<std::mutex> lk(g_tune_mtx);
        if (!g_tune_loaded && path) {
            std::ifstream f(path);
            std::string line;
            while (std::getline(f, line)) {
                std::istringstream ls(line);
                std::string k;
                int xc = 0, ty = 0;
                if (ls >> k >> xc >> ty && xc > 0) g_tune[k] = {xc, ty};
            }
        }
        g_tune_loaded = true;
        auto it = g_tune.find(key);
        if (it != g_tune.end() && (!tma || tile_height_fits(P, it->second.second))) {
            P->xchunk = it->second.first;
            if (tma) P->tile_y = it->second.second;
            return PROP_OK;
        }
    }
    std::vector<int> heights;
    if (!tma) heights = {P->tile_y};
    else if (fty) heights = {P->tile_y};
    else
        for (int ty : {16, 8, 32})
            if (tile_height_fits(P, ty)) heights.push_back(ty);
    const int NX = P->g.NX;
    std::vector<int> cand;
    for (int c : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48}) {
        const int xc = std::max(8, (NX + c - 1) / c);
        if (std::find(cand.begin(), cand.end(), xc) == cand.end()) cand.push_back(xc);
    }
    const int heuristic = P->xchunk, ty0 = P->tile_y;
    if (std::find(cand.begin(), cand.end(), heuristic) == cand.end()) cand.push_back(heuristic);
    float *s[9];
    for (int i = 0; i < 9; i++) s[i] = P->st[i];
    WP_TRY(zero_fields(P, s, nfields(P)));
    cudaEvent_t e0, e1;
    WP_CK(P, cudaEventCreate(&e0));
    WP_CK(P, cudaEventCreate(&e1));
    // time 3 steps of a candidate (after one untimed step: the first launch
    // of a variant loads its module)
    auto trial = [&](int ty, int xc, bool warm, float *ms) -> int {
        P->tile_y = ty;
        P->xchunk = xc;
        if (warm) WP_TRY(step_state(P, s, false));
        WP_CK(P, cudaEventRecord(e0, P->stream));
        for (int i = 0; i < 3; i++) WP_TRY(step_state(P, s, false));
        WP_CK(P, cudaEventRecord(e1, P->stream));
        WP_CK(P, cudaEventSynchronize(e1));
        WP_CK(P, cudaEventElapsedTime(ms, e0, e1));
        return PROP_OK;
    };
    struct Trial {
        float ms;
        int ty, xc;
    };
    std::vector<Trial> t;
    for (int ty : heights)
        for (int xc : cand) {
            float ms = 0.f;
            WP_TRY(trial(ty, xc, true, &ms));
            t.push_back({ms, ty, xc});
        }
    // the three fastest again, in two interleaved rounds: the choice is the
    // least total of the three timings (one pass alone can be off by a few
    // per cent, more than the differences among the leaders)
    std::sort(t.begin(), t.end(), [](const Trial &a, const Trial &b) { return a.ms < b.ms; });
    t.resize(std::min<size_t>(t.size(), 3));
    for (int round = 0; round < 2 && t.size() > 1; round++)
        for (auto &c : t) {
            float ms = 0.f;
            WP_TRY(trial(c.ty, c.xc, false, &ms));
            c.ms += ms;
        }
    const Trial win = *std::min_element(t.begin(), t.end(), [](const Trial &a, const Trial &b) { return a.ms < b.ms; });
    const int best = t.empty() ? heuristic : win.xc, best_ty = t.empty() ? ty0 : win.ty;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < 9; i++) P->st[i] = s[i];
    WP_TRY(zero_fields(P, s, nfields(P)));
    P->xchunk = best;
    P->tile_y = best_ty;
    std::lock_guard<std::mutex> lk(g_tune_mtx);
    g_tune[key] = {best, best_ty};
    if (path) {
        std::ofstream f(path, std::ios::app);
        f << key << ' ' << best << ' ' << best_ty << '\n';
    }
    return PROP_OK;
}

extern "C" int prop_tile_planes(const prop_t *P) { return P ? P->xchunk : 0; }
extern "C" int prop_tile_rows(const prop_t *P) { return P ? P->tile_y : 0; }

static int create_impl(prop_s *P, const prop_desc *d, const float *const *model)
{
    P->d = *d;
    const int so = d->space_order;
    if (d->kind != PROP_TTI && d->kind != PROP_ELASTIC && d->kind != PROP_ACOUSTIC && d->kind != PROP_ELASTIC2D)
        return wp_fail(P, PROP_EINVAL, "kind must be PROP_TTI, PROP_ELASTIC, PROP_ACOUSTIC or PROP_ELASTIC2D");
    if (d->kind == PROP_ELASTIC2D && d->ny != 1) return wp_fail(P, PROP_EINVAL, "PROP_ELASTIC2D needs ny = 1");
    if (d->tti_operator != 0 && (d->kind != PROP_TTI || d->tti_operator != 1))
        return wp_fail(P, PROP_EINVAL, "tti_operator must be 0, or 1 for PROP_TTI");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return wp_fail(P, PROP_EINVAL, "grid sizes must be >= 1");
    if (d->nbl < 0) return wp_fail(P, PROP_EINVAL, "nbl must be >= 0");
    if (!(d->h > 0.f) || !std::isfinite(d->h)) return wp_fail(P, PROP_EINVAL, "h must be > 0");
    if (so != 4 && so != 8 && so != 12 && so != 16) return wp_fail(P, PROP_EINVAL, "space_order must be 4, 8, 12 or 16");
    if (d->nt < 2) return wp_fail(P, PROP_EINVAL, "nt must be >= 2");
    if (d->snap_mode < 0 || d->snap_mode > 3) return wp_fail(P, PROP_EINVAL, "snap_mode out of range");
    if (d->ckpt_interval < 0) return wp_fail(P, PROP_EINVAL, "ckpt_interval must be >= 0");
    if (!model) return wp_fail(P, PROP_EINVAL, "model is NULL");
    const int nf = d->kind == PROP_TTI ? 5 : (d->kind == PROP_ACOUSTIC ? 1 : 3);
    for (int i = 0; i < nf; i++)
        if (!model[i]) return wp_fail(P, PROP_EINVAL, "model array is NULL");
    P->M = so / 2;
    GridDev &g = P->g;
    g.nbl = d->nbl;
    g.nby = d->kind == PROP_ELASTIC2D ? 0 : d->nbl;
    g.px = d->nx; g.py = d->ny; g.pz = d->nz;
    g.NX = d->nx + 2 * d->nbl; g.NY = d->ny + 2 * g.nby; g.NZ = d->nz + 2 * d->nbl;
    g.N = (long long)g.NX * g.NY * g.NZ;
    if (g.N >= (1LL << 32)) return wp_fail(P, PROP_EINVAL, "computational grid above 2^32 - 1 points");
    g.h = d->h; g.ih = 1.f / d->h;
    if (!fd_weights(P->M, P->w.c, P->w.b)) return wp_fail(P, PROP_EINVAL, "FD weights");
    d2_weights(P->M, P->w.d2);

    // model on the host for validation
    const size_t np = (size_t)d->nx * d->ny * d->nz;
    std::vector<std::vector<float>> hm(nf);
    for (int i = 0; i < nf; i++) {
        hm[i].resize(np);
        WP_CK(P, cudaMemcpy(hm[i].data(), model[i], np * sizeof(float), cudaMemcpyDefault));
    }
    double vmax = 0.0;
    for (size_t q = 0; q < np; q++) {
        const float vp = hm[0][q];
        if (!(vp > 0.f) || !std::isfinite(vp)) return wp_fail(P, PROP_EINVAL, "vp must be finite and > 0");
        if (d->kind == PROP_TTI) {
            const float e = hm[1][q], dl = hm[2][q];
            if (!std::isfinite(e) || !std::isfinite(dl) || !std::isfinite(hm[3][q]) || !std::isfinite(hm[4][q]))
                return wp_fail(P, PROP_EINVAL, "non-finite TTI parameter");
            if (e < dl) return wp_fail(P, PROP_EINVAL, "epsilon < delta somewhere (TTI stability needs eps >= delta)");
            if (1.0 + 2.0 * dl <= 0.0) return wp_fail(P, PROP_EINVAL, "1 + 2 delta must be > 0");
            vmax = std::max(vmax, 1000.0 * vp * sqrt(1.0 + 2.0 * e));
        } else if (d->kind == PROP_ACOUSTIC) {
            vmax = std::max(vmax, 1000.0 * vp);
        } else {
            const float vs = hm[1][q], rho = hm[2][q];
            if (!(vs >= 0.f) || !std::isfinite(vs)) return wp_fail(P, PROP_EINVAL, "vs must be finite and >= 0");
            if (!(rho > 0.f) || !std::isfinite(rho)) return wp_fail(P, PROP_EINVAL, "rho must be finite and > 0");
            if ((double)vp * vp < 2.0 * (double)vs * vs) return wp_fail(P, PROP_EINVAL, "lambda < 0 (vp^2 < 2 vs^2)");
            vmax = std::max(vmax, 1000.0 * vp);
        }
    }
    P->vmax = (float)vmax;
    const double dt = d->dt > 0.f ? (double)d->dt : 0.4 * d->h / vmax;
    g.dt = (float)dt;
    P->d.dt = g.dt;
    // CFL: vmax dt / h <= 2 / (sqrt(3) max|symbol|)
    // (acoustic: vmax dt / h <= 2 / sqrt(3 max|symbol of h^2 D2|); 2D: sqrt(2))
    const bool stag = d->kind == PROP_ELASTIC || d->kind == PROP_ELASTIC2D;
    const double ndim = d->kind == PROP_ELASTIC2D ? 2.0 : 3.0;
    const double lim = d->kind == PROP_ACOUSTIC ? 2.0 / sqrt(3.0 * symbol2_max(P->w.d2, P->M))
                                                : 2.0 / (sqrt(ndim) * symbol_max(stag ? P->w.b : P->w.c, P->M, stag));
    const double cour = vmax * dt / d->h;
    if (cour > lim) {
        char buf[200];
        snprintf(buf, sizeof buf, "dt = %g s gives Courant number %.4f above the stability bound %.4f", dt, cour, lim);
        return wp_fail(P, PROP_EUNSTABLE, buf);
    }
    g.cer = 0.015f;
    if (d->nbl > 0) {
        const double L = d->nbl * (double)d->h;
        const double vd = d->vdamp > 0.f ? (double)d->vdamp : vmax;
        g.sig0 = (float)(3.0 * vd / (2.0 * L) * log(1000.0));
    }
    // device model
    const size_t N = (size_t)g.N;
    float *phys = nullptr;
    WP_MALLOC(P, phys, np * sizeof(float), "model staging");
    std::unique_ptr<float, decltype(&cudaFree)> guard(phys, &cudaFree);
    auto upload = [&](int i, float *&dst, float scale, int mode) -> int {
        WP_MALLOC(P, dst, N * sizeof(float), "model");
        WP_CK(P, cudaMemcpyAsync(phys, hm[i].data(), np * sizeof(float), cudaMemcpyHostToDevice, P->stream));
        k_extend(P, phys, dst, scale, mode);
        return PROP_OK;
    };
    if (d->kind == PROP_TTI) {
        WP_TRY(upload(0, P->m, 1000.f, 1));
        WP_TRY(upload(1, P->eps, 1.f, 0));
        WP_TRY(upload(2, P->del, 1.f, 0));
        WP_TRY(upload(3, P->th, 1.f, 0));
        WP_TRY(upload(4, P->ph, 1.f, 0));
        WP_MALLOC(P, P->nrm[0], N * sizeof(float), "symmetry axis");
        WP_MALLOC(P, P->nrm[1], N * sizeof(float), "symmetry axis");
        k_normals(P);
    } else if (d->kind == PROP_ACOUSTIC) {
        WP_TRY(upload(0, P->m, 1000.f, 1));
        WP_MALLOC(P, P->acw, N * sizeof(float), "model");
        k_ratio(P, P->m, g.dt * g.dt, P->acw, (long long)N);
    } else {
        WP_TRY(upload(0, P->bu, 1.f, 0));    // vp  -> b      (k_lame)
        WP_TRY(upload(1, P->lam, 1.f, 0));   // vs  -> lambda
        WP_TRY(upload(2, P->mu, 1.f, 0));    // rho -> mu
        k_lame(P);
    }
    {
        const std::vector<float> tab = layer_tables(g, d->kind);
        WP_MALLOC(P, P->tab, tab.size() * sizeof(float), "layer tables");
        WP_CK(P, cudaMemcpy(P->tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
        g.tab = P->tab;
        int dev = 0, sms = 152;
        WP_CK(P, cudaGetDevice(&dev));
        WP_CK(P, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        P->xchunk = stencil_xchunk(g, sms);
    }
    for (int i = 0; i < nfields(P); i++) WP_MALLOC(P, P->st[i], N * sizeof(float), "state");
    WP_TRY(ensure_tmp(P, d->kind == PROP_TTI ? (d->tti_operator == 1 ? 14 : 8) : 0));
    WP_MALLOC(P, P->flag, sizeof(int), "flag");
    WP_CK(P, cudaMemsetAsync(P->flag, 0, sizeof(int), P->stream));
    WP_TRY(autotune_tiles(P));
    WP_CK(P, cudaMemsetAsync(P->flag, 0, sizeof(int), P->stream));
    WP_CK(P, cudaStreamSynchronize(P->stream));
    WP_CK(P, cudaGetLastError());
    return PROP_OK;
}

extern "C" int prop_create(const prop_desc *desc, const float *const *model, void *cuda_stream,
                           prop_t **out)
{
    if (!out) return wp_fail(nullptr, PROP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return wp_fail(nullptr, PROP_EINVAL, "desc is NULL");
    prop_s *P = new prop_s();
    P->stream = (cudaStream_t)cuda_stream;
    int rc = create_impl(P, desc, model);
    if (rc) {
        std::string m = P->err;
        free_all(P);
        delete P;
        tl_err = m;
        return rc;
    }
    *out = P;
    return PROP_OK;
}

extern "C" void prop_destroy(prop_t *P)
{
    if (!P) return;
    if (P->stream) cudaStreamSynchronize(P->stream);
    free_all(P);
    delete P;
}

extern "C" const char *prop_last_error(const prop_t *P)
{
    return P ? P->err.c_str() : tl_err.c_str();
}

extern "C" float prop_dt(const prop_t *P) { return P ? P->g.dt : 0.f; }

extern "C" int prop_grid_dims(const prop_t *P, int *dims, int *nf)
{
    if (!P) return wp_fail(nullptr, PROP_EINVAL, "NULL handle");
    if (dims) { dims[0] = P->g.NX; dims[1] = P->g.NY; dims[2] = P->g.NZ; }
    if (nf) *nf = nfields(P);
    return PROP_OK;
}

static int check_usable(prop_s *P)
{
    if (!P) return wp_fail(nullptr, PROP_EINVAL, "NULL handle");
    if (P->broken) return wp_fail(P, PROP_ESTATE, "handle unusable after an earlier CUDA error: " + P->err);
    return PROP_OK;
}
// start of a call that launches work: the launch count starts from zero
static int check_handle(prop_s *P)
{
    WP_TRY(check_usable(P));
    P->kern_launches = 0;
    return PROP_OK;
}

// end of a call: surface asynchronous errors and the NaN flag
static int finish(prop_s *P)
{
    WP_CK(P, cudaStreamSynchronize(P->stream));
    WP_CK(P, cudaGetLastError());
    prof_collect(P);
    int f = 0;
    WP_CK(P, cudaMemcpy(&f, P->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) WP_CK(P, cudaMemset(P->flag, 0, sizeof(int)));
    return wp_flag_status(P, f);
}

int wp_flag_status(prop_s *P, int f)
{
    // bit 8: the bounds-checking build (WAVEPROP_CHECK=1) skipped an access
    if (f & 8) return wp_fail(P, PROP_ECUDA, "device bounds check failed (an access was skipped)");
    if (f & 2) return wp_fail(P, PROP_ETIMEOUT, "a bounded device-side wait expired (TMA pipeline)");
    if (P->d.check_nan && (f & 1)) return wp_fail(P, PROP_EUNSTABLE, "NaN or Inf in the wavefield");
    return PROP_OK;
}

static int zero_fields(prop_s *P, float *const *f, int n)
{
    for (int i = 0; i < n; i++) WP_CK(P, cudaMemsetAsync(f[i], 0, sizeof(float) * P->g.N, P->stream));
    return PROP_OK;
}

// ---------------------------------------------------------------------------
// state access
// ---------------------------------------------------------------------------
extern "C" int prop_set_state(prop_t *P, const float *const *fields)
{
    WP_TRY(check_handle(P));
    WP_TRY(ensure_work(P));
    if (!fields) return wp_fail(P, PROP_EINVAL, "fields is NULL");
    for (int i = 0; i < nfields(P); i++) {
        if (!fields[i]) return wp_fail(P, PROP_EINVAL, "field pointer is NULL");
        WP_CK(P, cudaMemcpyAsync(P->st[i], fields[i], sizeof(float) * P->g.N, cudaMemcpyDefault, P->stream));
    }
    return finish(P);
}

extern "C" int prop_get_state(prop_t *P, float *const *fields)
{
    WP_TRY(check_handle(P));
    WP_TRY(ensure_work(P));
    if (!fields) return wp_fail(P, PROP_EINVAL, "fields is NULL");
    for (int i = 0; i < nfields(P); i++) {
        if (!fields[i]) return wp_fail(P, PROP_EINVAL, "field pointer is NULL");
        WP_CK(P, cudaMemcpyAsync(fields[i], P->st[i], sizeof(float) * P->g.N, cudaMemcpyDefault, P->stream));
    }
    return finish(P);
}

static int step_state(prop_s *P, float **s, bool adjoint)
{
    if (P->d.kind == PROP_TTI) {
        WP_TRY(tti_launch_step(P, s, adjoint, nullptr, nullptr, nullptr));
        std::swap(s[0], s[2]);
        std::swap(s[1], s[3]);
    } else if (P->d.kind == PROP_ACOUSTIC) {          // the transposed step is the same map
        WP_TRY(acu_launch_step(P, s, nullptr, nullptr));
        std::swap(s[0], s[1]);
    } else if (P->d.kind == PROP_ELASTIC2D) {
        if (adjoint) return wp_fail(P, PROP_EINVAL, "transposed state steps are not available for PROP_ELASTIC2D");
        WP_TRY(el2_launch(P, s, 1.f));
    } else {
        if (adjoint) WP_TRY(ensure_tmp(P, 9));
        WP_TRY(el_launch_step(P, s, adjoint));
    }
    prof_maybe_collect(P);
    return PROP_OK;
}

// capture two source-free steps of the current state buffers into a graph
// (on a private stream; the launches of step_state are recorded, not run),
// or reuse the one captured for the same buffers, direction and tiles
static bool step_graph_ready(prop_s *P, bool adjoint)
{
    const int nf = nfields(P);
    bool same = P->step_graph && P->graph_adj == (int)adjoint && P->graph_xc == P->xchunk &&
                P->graph_ty == P->tile_y;
    for (int i = 0; same && i < nf; i++) same = P->graph_st[i] == P->st[i];
    if (same) return true;
    if (P->step_graph) {
        cudaGraphExecDestroy(P->step_graph);
        P->step_graph = nullptr;
    }
    if (!P->graph_stream && cudaStreamCreateWithFlags(&P->graph_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        P->graph_stream = nullptr;
        return false;
    }
    if (adjoint && P->d.kind == PROP_ELASTIC && ensure_tmp(P, 9) != PROP_OK) return false;   // no allocation while capturing
    cudaStream_t own = P->stream;
    const bool was_broken = P->broken;
    const std::string was_err = P->err;
    float *s[9];
    for (int i = 0; i < 9; i++) s[i] = P->st[i];
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(P->graph_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        P->stream = P->graph_stream;
        const long long launches = P->kern_launches;
        ok = step_state(P, s, adjoint) == PROP_OK && step_state(P, s, adjoint) == PROP_OK;
        P->graph_launches = P->kern_launches - launches;
        P->kern_launches = launches;
        P->stream = own;
        ok = (cudaStreamEndCapture(P->graph_stream, &graph) == cudaSuccess) && ok;
    }
    for (int i = 0; ok && i < nf; i++) ok = s[i] == P->st[i];    // a pair restores the buffers
    if (ok) ok = cudaGraphInstantiate(&P->step_graph, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {                           // stay on direct launches; the handle is unaffected
        cudaGetLastError();
        P->step_graph = nullptr;
        P->broken = was_broken;
        P->err = was_err;
        return false;
    }
    P->graph_adj = (int)adjoint;
    P->graph_xc = P->xchunk;
    P->graph_ty = P->tile_y;
    for (int i = 0; i < 9; i++) P->graph_st[i] = P->st[i];
    return true;
}

extern "C" int prop_step(prop_t *P, int nsteps, int adjoint)
{
    WP_TRY(check_handle(P));
    WP_TRY(ensure_work(P));
    // TTI transposed steps differentiate zeta = C lam, which each step then
    // keeps up to date: form it once from the state
    if (adjoint && P->d.kind == PROP_TTI && nsteps > 0) k_tti_zeta(P, P->st[0], P->st[1], P->tmp[6], P->tmp[7]);
    if (nsteps < 0) return wp_fail(P, PROP_EINVAL, "nsteps < 0");
    int done = 0;
    if (nsteps >= 4 && !P->prof) {
        // pairs of steps replayed from a CUDA graph (a pair returns the
        // rotating state buffers of TTI and acoustic to their places)
        const char *env = getenv("WAVEPROP_GRAPHS");
        const bool off = env && !strcmp(env, "0"), required = env && !strcmp(env, "1");
        if (!off && !step_graph_ready(P, adjoint != 0) && required)
            return wp_fail(P, PROP_EINVAL, "prop_step: step graph could not be captured");
        if (!off && P->step_graph) {
            for (; done + 2 <= nsteps; done += 2) {
                WP_CK(P, cudaGraphLaunch(P->step_graph, P->stream));
                P->kern_launches += P->graph_launches;
            }
        }
    }
    for (int i = done; i < nsteps; i++) WP_TRY(step_state(P, P->st, adjoint != 0));
    return finish(P);
}

extern "C" int prop_kernel_time(const prop_t *P, double *ms, long long *launches)
{
    if (!P) return wp_fail(nullptr, PROP_EINVAL, "NULL handle");
    double t = 0.0;
    long long n = 0;
    for (int i = 0; i < 8; i++) { t += P->prof_ms[i]; n += P->prof_n[i]; }
    if (ms) *ms = t;
    if (launches) *launches = n;
    return PROP_OK;
}

// measurement hooks (waveprop_diag.h)
extern "C" int prop_profile(prop_t *P, int on)
{
    if (!P) return wp_fail(nullptr, PROP_EINVAL, "NULL handle");
    prof_collect(P);
    P->prof = on != 0;
    for (int i = 0; i < 8; i++) { P->prof_ms[i] = 0.0; P->prof_n[i] = 0; }
    return PROP_OK;
}
extern "C" int prop_kernel_stats(const prop_t *P, int id, double *ms, long long *n)
{
    if (!P || id < 0 || id >= 8) return wp_fail(nullptr, PROP_EINVAL, "bad handle or id");
    if (ms) *ms = P->prof_ms[id];
    if (n) *n = P->prof_n[id];
    return PROP_OK;
}
extern "C" long long prop_last_launches(const prop_t *P) { return P ? P->kern_launches : 0; }
// failure-path self-test: a device wait that nothing completes gives up after
// `seconds` and the call returns PROP_ETIMEOUT (the handle then reports
// PROP_ESTATE, as after any expired wait); the context stays usable
extern "C" int prop_selftest_wait(prop_t *P, float seconds)
{
    WP_TRY(check_handle(P));
    WP_TRY(wait_probe_launch(P, seconds));
    return finish(P);
}

// ---------------------------------------------------------------------------
// forward modelling with optional saving of forward wavefields
// ---------------------------------------------------------------------------
struct Geometry {
    SparseDev S, R;
    ~Geometry() { sp_free(&S); sp_free(&R); }
};

// levels 1 .. ckpt_span are recomputed from checkpoints; the levels above
// it (FP32 checkpoints only) are kept in full in the tail buffer
static int ckpt_span(const prop_s *P) { return P->d.nt - 1 - P->tail_T; }

static int ckpt_K(const prop_s *P)
{
    const int span = std::max(1, ckpt_span(P));
    int K = P->d.ckpt_interval;
    if (K <= 0) K = (int)ceil(sqrt((double)span));
    return std::max(1, std::min(K, span));
}
static int ckpt_J(const prop_s *P)
{
    const int K = ckpt_K(P), span = ckpt_span(P);
    return span > 0 ? (span + K - 1) / K : 0;
}

// fields per stored forward level: TTI p, r; acoustic u; elastic on the
// TMA-fed passes only the velocities (the imaging reads the strain of
// v^{k+1} and the face products (v^{k+1}/g - v^k)/b_avg), else all 9
static size_t snap_fields(const prop_s *P)
{
    switch (P->d.kind) {
    case PROP_TTI: return 2;
    case PROP_ACOUSTIC: return 1;
    case PROP_ELASTIC2D: return 5;
    default: return tma_usable(P) ? 3 : 9;
    }
}

// tail of full FP32 levels for FP32 checkpoints (TTI, acoustic): as many
// levels as fit in 80 % of the free device memory left after the
// checkpoints and the segment buffer; WAVEPROP_CKPT_TAIL caps it (0: none)
static int choose_tail(prop_s *P)
{
    P->tail_T = 0;
    if (P->d.snap_mode != SNAP_CKPT_FP32 || P->no_tail || P->aniso ||
        (P->d.kind != PROP_TTI && P->d.kind != PROP_ACOUSTIC))
        return 0;
    const char *e = getenv("WAVEPROP_CKPT_TAIL");
    long cap = e ? atol(e) : (long)P->d.nt;
    if (cap <= 0) return 0;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const size_t N = (size_t)P->g.N, level = snap_fields(P) * N * sizeof(float);
    const size_t ck = (size_t)nfields(P) * N * sizeof(float);
    const int nt = P->d.nt;
    int T = (int)std::min<long>(cap, nt - 1);
    // shrink until tail + checkpoints + segment buffer fit the budget
    const double budget = 0.8 * (double)fr - (double)(1ull << 30);
    for (; T > 0; T = T * 15 / 16) {
        P->tail_T = T;
        const double need = (double)T * level + (double)ckpt_J(P) * ck + (double)(ckpt_K(P) + 1) * level;
        if (need <= budget) break;
    }
    P->tail_T = std::max(0, T);
    return P->tail_T;
}

static int alloc_saves(prop_s *P)
{
    free_snaps(P);
    choose_tail(P);
    const size_t N = (size_t)P->g.N;
    const int nt = P->d.nt, K = ckpt_K(P);
    const int J = ckpt_J(P);                 // checkpoints / segments
    const int cf = nfields(P);               // fields per checkpoint
    switch (P->d.snap_mode) {
    case SNAP_FULL_FP32: {
        // TTI: u^k, k = 1..nt-1 (p, r); acoustic: u^k, k = 1..nt-1;
        // elastic: X^k, k = 0..nt-1 (9 fields)
        const size_t slots = P->d.kind != PROP_ELASTIC ? (size_t)(nt - 1) : (size_t)nt;
        P->snap_bytes = slots * snap_fields(P) * N * sizeof(float);
        WP_MALLOC(P, P->snap, P->snap_bytes, "full FP32 wavefield storage");
        break;
    }
    case SNAP_CKPT_FP32:
        P->snap_bytes = (size_t)std::max(J, 1) * cf * N * sizeof(float);
        WP_MALLOC(P, P->snap, P->snap_bytes, "FP32 checkpoints");
        if (P->tail_T > 0) {
            P->tail_bytes = (size_t)P->tail_T * snap_fields(P) * N * sizeof(float);
            WP_MALLOC(P, P->tail, P->tail_bytes, "full FP32 tail of the checkpointed run");
        }
        break;
    default:
        P->snap16_bytes = (size_t)J * cf * N * sizeof(uint16_t);
        WP_MALLOC(P, P->snap16, P->snap16_bytes, "16-bit checkpoints");
        WP_MALLOC(P, P->snap_scale, sizeof(float) * J * cf + 1024 * sizeof(float), "checkpoint scales");
        break;
    }
    if (P->d.snap_mode != SNAP_FULL_FP32) {
        // TTI: levels n0+1 .. n0+K of a segment and (slot K) the checkpoint
        // level n0 itself (eps/delta imaging); elastic: levels n0 .. n0+K
        const size_t slots = (size_t)K + 1;
        P->seg_bytes = slots * snap_fields(P) * N * sizeof(float);
        WP_MALLOC(P, P->seg, P->seg_bytes, "recompute segment buffer");
    }
    return PROP_OK;
}

static float *snap_slot(prop_s *P, size_t slot)
{
    return P->snap + slot * snap_fields(P) * (size_t)P->g.N;
}
static float *seg_slot(prop_s *P, size_t slot)
{
    return P->seg + slot * snap_fields(P) * (size_t)P->g.N;
}

static int save_checkpoint(prop_s *P, int j, float *const *s)
{
    const size_t N = (size_t)P->g.N;
    const int cf = nfields(P);
    const size_t nscale = (size_t)ckpt_J(P) * cf;   // scales, then 1024 partials
    for (int f = 0; f < cf; f++) {
        const size_t slot = (size_t)j * cf + f;
        if (P->d.snap_mode == SNAP_CKPT_FP32)
            WP_CK(P, cudaMemcpyAsync(P->snap + slot * N, s[f], N * sizeof(float), cudaMemcpyDeviceToDevice, P->stream));
        else
            k_snap_encode(P, s[f], (long long)N, P->snap16 + slot * N, P->snap_scale + slot,
                          P->d.snap_mode == SNAP_CKPT_BF16, P->snap_scale + nscale);
    }
    return PROP_OK;
}
static int load_checkpoint(prop_s *P, int j, float *const *s)
{
    const size_t N = (size_t)P->g.N;
    const int cf = nfields(P);
    for (int f = 0; f < cf; f++) {
        const size_t slot = (size_t)j * cf + f;
        if (P->d.snap_mode == SNAP_CKPT_FP32)
            WP_CK(P, cudaMemcpyAsync(s[f], P->snap + slot * N, N * sizeof(float), cudaMemcpyDeviceToDevice, P->stream));
        else
            k_snap_decode(P, P->snap16 + slot * N, (long long)N, P->snap_scale + slot,
                          P->d.snap_mode == SNAP_CKPT_BF16, s[f]);
    }
    return PROP_OK;
}

// inject q^n into the new level of state s (after the step)
static void inject_src(prop_s *P, const SparseDev &S, const float *wav, int n, float *const *s)
{
    const int nt = P->d.nt;
    if (P->d.kind == PROP_TTI)
        sp_inject(P, &S, wav, nt, n, P->g.dt * P->g.dt, 1, s[0], s[1], nullptr, nullptr, nullptr);
    else if (P->d.kind == PROP_ACOUSTIC)
        sp_inject(P, &S, wav, nt, n, P->g.dt * P->g.dt, 1, s[0], nullptr, nullptr, nullptr, nullptr);
    else if (P->d.kind == PROP_ELASTIC2D)
        sp_inject(P, &S, wav, nt, n, P->g.dt, 0, s[2], s[3], nullptr, nullptr, nullptr);
    else
        sp_inject(P, &S, wav, nt, n, P->g.dt, 0, s[3], s[4], s[5], nullptr, nullptr);
}
static void record_rec(prop_s *P, const SparseDev &R, float *const *s, float *col)
{
    if (P->d.kind == PROP_TTI || P->d.kind == PROP_ACOUSTIC) sp_record(P, &R, s[0], nullptr, nullptr, 1.f, col);
    else if (P->d.kind == PROP_ELASTIC2D) sp_record(P, &R, s[2], s[3], nullptr, 1.f, col);
    else sp_record(P, &R, s[3], s[4], s[5], 1.f, col);
}

// One forward step n of state s (record already done).  TTI/acoustic
// pointer rotation is applied so that s[0] (TTI: s[0..1]) hold the new level
// afterwards.
static int fwd_step(prop_s *P, float **s, const SparseDev &S, const float *wav, int n)
{
    if (P->d.kind == PROP_TTI) {
        WP_TRY(tti_launch_step(P, s, false, nullptr, nullptr, nullptr));
        std::swap(s[0], s[2]);
        std::swap(s[1], s[3]);
    } else if (P->d.kind == PROP_ACOUSTIC) {
        WP_TRY(acu_launch_step(P, s, nullptr, nullptr));
        std::swap(s[0], s[1]);
    } else if (P->d.kind == PROP_ELASTIC2D) {
        WP_TRY(el2_launch(P, s, 1.f));
    } else {
        WP_TRY(el_launch_step(P, s, false));
    }
    inject_src(P, S, wav, n, s);
    prof_maybe_collect(P);
    return PROP_OK;
}

// store level `lvl` (state s holds level lvl) in full storage
static int store_full(prop_s *P, float *const *s, int lvl)
{
    const size_t N = (size_t)P->g.N;
    if (P->d.kind != PROP_ELASTIC) {
        if (lvl < 1 || lvl > P->d.nt - 1) return PROP_OK;
        float *d = snap_slot(P, lvl - 1);
        for (size_t f = 0; f < snap_fields(P); f++)
            WP_CK(P, cudaMemcpyAsync(d + f * N, s[f], N * 4, cudaMemcpyDeviceToDevice, P->stream));
    } else {
        if (lvl < 0 || lvl > P->d.nt - 1) return PROP_OK;
        float *d = snap_slot(P, lvl);
        for (size_t f = 0; f < snap_fields(P); f++)
            WP_CK(P, cudaMemcpyAsync(d + f * N, s[f], N * 4, cudaMemcpyDeviceToDevice, P->stream));
    }
    return PROP_OK;
}

// forward time loop; stage [nt][nrec]; save: keep wavefields per snap_mode
static int run_forward(prop_s *P, const Geometry &G, const float *wav, float *stage, bool save)
{
    const int nt = P->d.nt, K = ckpt_K(P);
    float *s[9];
    for (int i = 0; i < 9; i++) s[i] = P->st[i];
    WP_TRY(zero_fields(P, s, nfields(P)));
    const bool full = save && P->d.snap_mode == SNAP_FULL_FP32;
    const bool ckpt = save && !full;
    if (full && P->d.kind == PROP_ELASTIC) WP_TRY(store_full(P, s, 0));
    const int span = ckpt_span(P), L0 = nt - P->tail_T;   // tail: levels L0 .. nt-1
    const size_t tl = snap_fields(P) * (size_t)P->g.N;
    for (int n = 0; n < nt; n++) {
        record_rec(P, G.R, s, stage + (size_t)n * G.R.n);
        if (ckpt && n % K == 0 && n < span) WP_TRY(save_checkpoint(P, n / K, s));
        WP_TRY(fwd_step(P, s, G.S, wav, n));
        if (full) WP_TRY(store_full(P, s, n + 1));
        if (ckpt && P->tail_T > 0 && n + 1 >= L0 && n + 1 <= nt - 1) {
            float *d = P->tail + (size_t)(n + 1 - L0) * tl;
            for (size_t f = 0; f < snap_fields(P); f++)
                WP_CK(P, cudaMemcpyAsync(d + f * P->g.N, s[f], P->g.N * 4, cudaMemcpyDeviceToDevice, P->stream));
        }
    }
    // the final state, in st[] order, for prop_get_state (buffers permuted)
    for (int i = 0; i < nfields(P); i++) P->st[i] = s[i];
    return PROP_OK;
}

static int build_geometry(prop_s *P, Geometry &G, const float *src, int nsrc, const float *rec, int nrec)
{
    if (nsrc < 1 || nrec < 1) return wp_fail(P, PROP_EINVAL, "nsrc and nrec must be >= 1");
    if (!src || !rec) return wp_fail(P, PROP_EINVAL, "coordinates are NULL");
    std::vector<float> hs((size_t)nsrc * 3), hr((size_t)nrec * 3);
    WP_CK(P, cudaMemcpy(hs.data(), src, hs.size() * 4, cudaMemcpyDefault));
    WP_CK(P, cudaMemcpy(hr.data(), rec, hr.size() * 4, cudaMemcpyDefault));
    WP_TRY(sp_build(P, hs.data(), nsrc, nullptr, &G.S));
    WP_TRY(sp_build(P, hr.data(), nrec, nullptr, &G.R));
    return PROP_OK;
}

static int forward_impl(prop_s *P, const float *wavelet, const float *src, int nsrc,
                        const float *rec, int nrec, float *traces, bool save)
{
    WP_TRY(check_handle(P));
    if (!wavelet || !traces) return wp_fail(P, PROP_EINVAL, "wavelet or traces is NULL");
    if (save && P->d.kind == PROP_ELASTIC2D)
        return wp_fail(P, PROP_EINVAL, "gradients and saved forward runs are not available for PROP_ELASTIC2D");
    WP_TRY(ensure_work(P));
    Geometry G;
    WP_TRY(build_geometry(P, G, src, nsrc, rec, nrec));
    const int nt = P->d.nt;
    DevBuf wbuf, stage, tr;
    const float *wav = nullptr;
    WP_TRY(dev_in(P, wavelet, (size_t)nsrc * nt, wbuf, &wav));
    WP_TRY(wp_malloc(P, &stage.p, sizeof(float) * (size_t)nt * nrec, "trace staging"));
    WP_TRY(wp_malloc(P, &tr.p, sizeof(float) * (size_t)nt * nrec, "traces"));
    if (save) {
        WP_TRY(alloc_saves(P));
        if (P->d.kind == PROP_ELASTIC) WP_TRY(ensure_tmp(P, 15));
    }
    WP_TRY(run_forward(P, G, wav, (float *)stage.p, save));
    sp_transpose(P, (const float *)stage.p, (float *)tr.p, nrec, nt);
    WP_TRY(copy_out(P, traces, (const float *)tr.p, (size_t)nt * nrec));
    if (save) {
        P->saved = true;
        P->saved_nsrc = nsrc;
        P->saved_nrec = nrec;
        P->saved_src.resize((size_t)nsrc * 3);
        P->saved_rec.resize((size_t)nrec * 3);
        P->saved_wav.resize((size_t)nsrc * nt);
        WP_CK(P, cudaMemcpyAsync(P->saved_src.data(), src, (size_t)nsrc * 12, cudaMemcpyDefault, P->stream));
        WP_CK(P, cudaMemcpyAsync(P->saved_rec.data(), rec, (size_t)nrec * 12, cudaMemcpyDefault, P->stream));
        WP_CK(P, cudaMemcpyAsync(P->saved_wav.data(), wav, (size_t)nsrc * nt * 4, cudaMemcpyDefault, P->stream));
    }
    return finish(P);
}

extern "C" int prop_forward(prop_t *P, const float *wavelet, const float *src_xyz, int nsrc,
                            const float *rec_xyz, int nrec, float *traces)
{
    return forward_impl(P, wavelet, src_xyz, nsrc, rec_xyz, nrec, traces, false);
}

extern "C" int prop_forward_saved(prop_t *P, const float *wavelet, const float *src_xyz, int nsrc,
                                  const float *rec_xyz, int nrec, float *traces)
{
    int rc = forward_impl(P, wavelet, src_xyz, nsrc, rec_xyz, nrec, traces, true);
    if (rc && P) free_snaps(P);
    return rc;
}

// ---------------------------------------------------------------------------
// adjoint sweeps
// ---------------------------------------------------------------------------
// inject residual column k (traces [nrec][nt]) into the adjoint state
static void inject_resid(prop_s *P, const Geometry &G, const float *res, int k, float *const *a,
                         const float *img_p, float *grad)
{
    const int nt = P->d.nt;
    if (P->d.kind == PROP_TTI)   // also keeps zeta = C lam (tmp[6], tmp[7]) in step
        sp_inject(P, &G.R, res, nt, k, 1.f, 3, a[0], P->tmp[6], P->tmp[7], grad ? img_p : nullptr, grad);
    else if (P->d.kind == PROP_ACOUSTIC)
        sp_inject(P, &G.R, res, nt, k, 1.f, 1, a[0], nullptr, nullptr, grad ? img_p : nullptr, grad);
    else
        sp_inject(P, &G.R, res, nt, k, 1.f, 0, a[3], a[4], a[5], nullptr, nullptr);
}
// adjoint source output qbar^{k-1} from the adjoint state at level k
static void sample_src(prop_s *P, const Geometry &G, float *const *a, float *col)
{
    if (P->d.kind == PROP_TTI) sp_record(P, &G.S, a[0], a[1], nullptr, P->g.dt * P->g.dt, col);
    else if (P->d.kind == PROP_ACOUSTIC) sp_record(P, &G.S, a[0], nullptr, nullptr, P->g.dt * P->g.dt, col);
    else sp_record(P, &G.S, a[3], a[4], a[5], P->g.dt, col);
}

// TTI adjoint sweep.  grad != NULL: imaging with forward wavefields.
static int tti_sweep(prop_s *P, const Geometry &G, const float *res, const float *wav,
                     float *srcstage, float *const *g3)
{
    // g3: NULL (adjoint modelling), {dJ/dm} or, with P->aniso,
    // {dJ/dm, dJ/deps, dJ/ddelta, dJ/dn (3 components)}
    float *grad = g3 ? g3[0] : nullptr;
    const bool aniso = g3 && P->aniso;
    const int nt = P->d.nt;
    const size_t N = (size_t)P->g.N;
    WP_TRY(ensure_ast(P));
    if (aniso) WP_TRY(ensure_tmp(P, P->d.tti_operator == 1 ? 20 : 14));
    float *a[4] = {P->ast[0], P->ast[1], P->ast[2], P->ast[3]};
    WP_TRY(zero_fields(P, a, 4));
    WP_TRY(zero_fields(P, P->tmp + 6, 2));   // zeta = C lam of the zero state
    if (srcstage) WP_CK(P, cudaMemsetAsync(srcstage, 0, sizeof(float) * (size_t)nt * G.S.n, P->stream));
    auto adj_iter = [&](int k, const float *up, const float *ur) -> int {
        WP_TRY(tti_launch_step(P, a, true, up, ur, grad));
        std::swap(a[0], a[2]);
        std::swap(a[1], a[3]);
        inject_resid(P, G, res, k, a, up, grad);
        if (srcstage) sample_src(P, G, a, srcstage + (size_t)(k - 1) * G.S.n);
        prof_maybe_collect(P);
        return PROP_OK;
    };
    // eps/delta/axis imaging: lam^k (a[0], a[1] after the step and the
    // residual; zeta = C lam^k in tmp[6], tmp[7]) with the forward level k-1
    // (level 0 is zero: no term for k = 1)
    auto aniso_iter = [&](int k, const float *u1) -> int {
        if (!aniso || k < 2) return PROP_OK;
        if (tma_usable(P)) return tti_image_aniso_tma(P, u1, u1 + N, a[0], a[1], g3[1], g3[2], g3 + 3);
        return tti_image_aniso_fast(P, u1, u1 + N, a[0], a[1], g3[1], g3[2], g3 + 3);
    };
    if (!grad) {
        for (int k = nt - 1; k >= 1; k--) WP_TRY(adj_iter(k, nullptr, nullptr));
        return PROP_OK;
    }
    if (P->d.snap_mode == SNAP_FULL_FP32) {
        for (int k = nt - 1; k >= 1; k--) {
            const float *u = snap_slot(P, k - 1);
            WP_TRY(adj_iter(k, u, u + N));
            if (k >= 2) WP_TRY(aniso_iter(k, snap_slot(P, k - 2)));
        }
        return PROP_OK;
    }
    const int K = ckpt_K(P), J = ckpt_J(P), span = ckpt_span(P), L0 = nt - P->tail_T;
    // the tail: levels kept in full (no eps/delta/axis imaging here: the tail
    // is not used for prop_gradient_aniso)
    for (int k = nt - 1; k >= L0; k--) {
        const float *u = P->tail + (size_t)(k - L0) * 2 * N;
        WP_TRY(adj_iter(k, u, u + N));
    }
    float *s[4] = {P->st[0], P->st[1], P->st[2], P->st[3]};
    for (int j = J - 1; j >= 0; j--) {
        const int n0 = j * K, E = std::min((j + 1) * K, span);
        // restore level n0 and recompute levels n0+1..E
        float *f[4] = {P->st[0], P->st[1], P->st[2], P->st[3]};
        for (int i = 0; i < 4; i++) s[i] = f[i];
        WP_TRY(load_checkpoint(P, j, s));
        if (aniso) {                            // level n0 into the extra slot K
            WP_CK(P, cudaMemcpyAsync(seg_slot(P, K), s[0], N * 4, cudaMemcpyDeviceToDevice, P->stream));
            WP_CK(P, cudaMemcpyAsync(seg_slot(P, K) + N, s[1], N * 4, cudaMemcpyDeviceToDevice, P->stream));
        }
        for (int n = n0; n < E; n++) {
            WP_TRY(fwd_step(P, s, G.S, wav, n));
            float *d = seg_slot(P, n - n0);     // level n+1
            WP_CK(P, cudaMemcpyAsync(d, s[0], N * 4, cudaMemcpyDeviceToDevice, P->stream));
            WP_CK(P, cudaMemcpyAsync(d + N, s[1], N * 4, cudaMemcpyDeviceToDevice, P->stream));
        }
        for (int k = E; k >= n0 + 1; k--) {
            const float *u = seg_slot(P, k - n0 - 1);
            WP_TRY(adj_iter(k, u, u + N));
            WP_TRY(aniso_iter(k, k - 1 > n0 ? seg_slot(P, k - n0 - 2) : seg_slot(P, K)));
        }
    }
    return PROP_OK;
}

// acoustic adjoint sweep.  grad != NULL: imaging with the forward wavefield
// of the same level (lam^k pairs with u^k: -u^k (dt^2 L lam^{k+1} + R^T r^k) / m)
static int ac_sweep(prop_s *P, const Geometry &G, const float *res, const float *wav,
                    float *srcstage, float *grad)
{
    const int nt = P->d.nt;
    WP_TRY(ensure_ast(P));
    float *a[2] = {P->ast[0], P->ast[1]};
    WP_TRY(zero_fields(P, a, 2));
    if (srcstage) WP_CK(P, cudaMemsetAsync(srcstage, 0, sizeof(float) * (size_t)nt * G.S.n, P->stream));
    auto adj_iter = [&](int k, const float *u) -> int {
        WP_TRY(acu_launch_step(P, a, u, grad));   // a[1] <- lam^k
        std::swap(a[0], a[1]);
        inject_resid(P, G, res, k, a, u, grad);
        if (srcstage) sample_src(P, G, a, srcstage + (size_t)(k - 1) * G.S.n);
        prof_maybe_collect(P);
        return PROP_OK;
    };
    if (!grad) {
        for (int k = nt - 1; k >= 1; k--) WP_TRY(adj_iter(k, nullptr));
        return PROP_OK;
    }
    if (P->d.snap_mode == SNAP_FULL_FP32) {
        for (int k = nt - 1; k >= 1; k--) WP_TRY(adj_iter(k, snap_slot(P, k - 1)));
        return PROP_OK;
    }
    const size_t N = (size_t)P->g.N;
    const int K = ckpt_K(P), J = ckpt_J(P), span = ckpt_span(P), L0 = nt - P->tail_T;
    for (int k = nt - 1; k >= L0; k--) WP_TRY(adj_iter(k, P->tail + (size_t)(k - L0) * N));
    for (int j = J - 1; j >= 0; j--) {
        const int n0 = j * K, E = std::min((j + 1) * K, span);
        // restore level n0 and recompute levels n0+1..E (slot i: level n0+1+i)
        float *s[2] = {P->st[0], P->st[1]};
        WP_TRY(load_checkpoint(P, j, s));
        for (int n = n0; n < E; n++) {
            WP_TRY(fwd_step(P, s, G.S, wav, n));
            WP_CK(P, cudaMemcpyAsync(seg_slot(P, n - n0), s[0], N * 4, cudaMemcpyDeviceToDevice, P->stream));
        }
        for (int k = E; k >= n0 + 1; k--) WP_TRY(adj_iter(k, seg_slot(P, k - n0 - 1)));
    }
    return PROP_OK;
}

// 2D elastic adjoint modelling in the variables (b_avg vbar, g C tbar): the
// forward passes with dt -> -dt; residuals enter as g (2 lambda + 2 mu) r on
// xx and zz, the source side reads dt (u_xx + u_zz) / (g (2 lambda + 2 mu))
static int el2_sweep(prop_s *P, const Geometry &G, const float *res, float *srcstage)
{
    const int nt = P->d.nt;
    WP_TRY(ensure_ast(P));
    float *a[5];
    for (int i = 0; i < 5; i++) a[i] = P->ast[i];
    WP_TRY(zero_fields(P, a, 5));
    if (srcstage) WP_CK(P, cudaMemsetAsync(srcstage, 0, sizeof(float) * (size_t)nt * G.S.n, P->stream));
    for (int k = nt - 1; k >= 1; k--) {
        WP_TRY(el2_launch(P, a, -1.f));
        sp_inject(P, &G.R, res, nt, k, 1.f, 4, a[2], a[3], nullptr, nullptr, nullptr);
        if (srcstage)
            sp_record_trace_s(P, &G.S, a[2], a[3], nullptr, P->g.dt, srcstage + (size_t)(k - 1) * G.S.n);
        prof_maybe_collect(P);
    }
    return PROP_OK;
}

// elastic adjoint sweep; g3 != NULL: gradient (lambda, mu, b) on the computational grid
static int el_sweep(prop_s *P, const Geometry &G, const float *res, const float *wav,
                    float *srcstage, float *const *g3)
{
    const int nt = P->d.nt;
    const size_t N = (size_t)P->g.N;
    WP_TRY(ensure_ast(P));
    WP_TRY(ensure_tmp(P, g3 ? 15 : 9));
    float *a[9];
    for (int i = 0; i < 9; i++) a[i] = P->ast[i];
    WP_TRY(zero_fields(P, a, 9));
    if (srcstage) WP_CK(P, cudaMemsetAsync(srcstage, 0, sizeof(float) * (size_t)nt * G.S.n, P->stream));
    auto after = [&](int k) {
        if (k >= 1) {
            inject_resid(P, G, res, k, a, nullptr, nullptr);
            if (srcstage) sample_src(P, G, a, srcstage + (size_t)(k - 1) * G.S.n);
        }
        prof_maybe_collect(P);
    };
    if (!g3) {
        // adjoint modelling in s = C tbar: residuals enter as (3 lambda + 2 mu) w r,
        // the source side reads dt P tr(s) / (3 lambda + 2 mu)
        for (int k = nt - 1; k >= 1; k--) {
            WP_TRY(el_step_adjoint_u(P, a));
            sp_inject(P, &G.R, res, nt, k, 1.f, 2, a[3], a[4], a[5], nullptr, nullptr);
            if (srcstage)
                sp_record_trace_s(P, &G.S, a[3], a[4], a[5], P->g.dt, srcstage + (size_t)(k - 1) * G.S.n);
            prof_maybe_collect(P);
        }
        return PROP_OK;
    }
    // k = nt-1: transposed step of a zero state, then the last residual sample
    WP_TRY(zero_fields(P, P->tmp + 9, 6));      // edge and face product sums
    WP_TRY(el_launch_step(P, a, true));
    after(nt - 1);
    const int sf = (int)snap_fields(P);
    auto xs = [&](float *base, const float **out) {
        for (int f = 0; f < 9; f++) out[f] = f < sf ? base + f * N : nullptr;
    };
    if (P->d.snap_mode == SNAP_FULL_FP32) {
        for (int k = nt - 2; k >= 0; k--) {
            const float *x0[9], *x1[9];
            xs(snap_slot(P, k), x0);
            xs(snap_slot(P, k + 1), x1);
            WP_TRY(el_launch_adj_grad(P, a, x0, x1, g3));
            after(k);
        }
        return el_grad_gather(P, g3);
    }
    const int K = ckpt_K(P), J = (nt - 1 + K - 1) / K;
    for (int j = J - 1; j >= 0; j--) {
        const int n0 = j * K, E = std::min((j + 1) * K, nt - 1);
        float *s[9];
        for (int i = 0; i < 9; i++) s[i] = P->st[i];
        WP_TRY(load_checkpoint(P, j, s));
        for (int f = 0; f < sf; f++)
            WP_CK(P, cudaMemcpyAsync(seg_slot(P, 0) + f * N, s[f], N * 4, cudaMemcpyDeviceToDevice, P->stream));
        for (int n = n0; n < E; n++) {
            WP_TRY(fwd_step(P, s, G.S, wav, n));
            for (int f = 0; f < sf; f++)
                WP_CK(P, cudaMemcpyAsync(seg_slot(P, n + 1 - n0) + f * N, s[f], N * 4,
                                         cudaMemcpyDeviceToDevice, P->stream));
        }
        for (int k = E - 1; k >= n0; k--) {
            const float *x0[9], *x1[9];
            xs(seg_slot(P, k - n0), x0);
            xs(seg_slot(P, k + 1 - n0), x1);
            WP_TRY(el_launch_adj_grad(P, a, x0, x1, g3));
            after(k);
        }
    }
    return el_grad_gather(P, g3);
}

extern "C" int prop_adjoint(prop_t *P, const float *traces_in, const float *rec_xyz, int nrec,
                            const float *src_xyz, int nsrc, float *src_out)
{
    WP_TRY(check_handle(P));
    if (!traces_in || !src_out) return wp_fail(P, PROP_EINVAL, "traces_in or src_out is NULL");
    WP_TRY(ensure_work(P));
    Geometry G;
    WP_TRY(build_geometry(P, G, src_xyz, nsrc, rec_xyz, nrec));
    const int nt = P->d.nt;
    DevBuf rbuf, stage, out;
    const float *res = nullptr;
    WP_TRY(dev_in(P, traces_in, (size_t)nrec * nt, rbuf, &res));
    WP_TRY(wp_malloc(P, &stage.p, sizeof(float) * (size_t)nt * nsrc, "source staging"));
    WP_TRY(wp_malloc(P, &out.p, sizeof(float) * (size_t)nt * nsrc, "source output"));
    if (P->d.kind == PROP_TTI) WP_TRY(tti_sweep(P, G, res, nullptr, (float *)stage.p, nullptr));
    else if (P->d.kind == PROP_ACOUSTIC) WP_TRY(ac_sweep(P, G, res, nullptr, (float *)stage.p, nullptr));
    else if (P->d.kind == PROP_ELASTIC2D) WP_TRY(el2_sweep(P, G, res, (float *)stage.p));
    else WP_TRY(el_sweep(P, G, res, nullptr, (float *)stage.p, nullptr));
    sp_transpose(P, (const float *)stage.p, (float *)out.p, nsrc, nt);
    WP_TRY(copy_out(P, src_out, (const float *)out.p, (size_t)nt * nsrc));
    return finish(P);
}

// backward pass with the saved forward run
static int backward_impl(prop_s *P, const float *resid, float *grad, float *src_grad, double *misfit_unused)
{
    (void)misfit_unused;
    if (!P->saved) return wp_fail(P, PROP_ESTATE, "prop_backward needs a preceding prop_forward_saved");
    WP_TRY(ensure_work(P));
    const int nt = P->d.nt, nsrc = P->saved_nsrc, nrec = P->saved_nrec;
    Geometry G;
    WP_TRY(sp_build(P, P->saved_src.data(), nsrc, nullptr, &G.S));
    WP_TRY(sp_build(P, P->saved_rec.data(), nrec, nullptr, &G.R));
    DevBuf rbuf, wbuf, stage, out, gbuf, gphys;
    const float *res = nullptr;
    WP_TRY(dev_in(P, resid, (size_t)nrec * nt, rbuf, &res));
    WP_TRY(wp_malloc(P, &wbuf.p, sizeof(float) * (size_t)nsrc * nt, "wavelet"));
    WP_CK(P, cudaMemcpyAsync(wbuf.p, P->saved_wav.data(), sizeof(float) * (size_t)nsrc * nt,
                             cudaMemcpyHostToDevice, P->stream));
    if (src_grad) {
        WP_TRY(wp_malloc(P, &stage.p, sizeof(float) * (size_t)nt * nsrc, "source staging"));
        WP_TRY(wp_malloc(P, &out.p, sizeof(float) * (size_t)nt * nsrc, "source output"));
    }
    // computational-grid accumulators and physical outputs: TTI m (+ eps,
    // delta and the three dJ/dn components that become theta, phi); elastic
    // lambda, mu, b
    const bool aniso = P->d.kind == PROP_TTI && P->aniso;
    const int ng = P->d.kind == PROP_TTI ? (aniso ? 6 : 1) : (P->d.kind == PROP_ACOUSTIC ? 1 : 3),
              nout = aniso ? 5 : ng;
    const size_t N = (size_t)P->g.N, np = (size_t)P->g.px * P->g.py * P->g.pz;
    float *g3[6] = {};
    if (grad) {
        WP_TRY(wp_malloc(P, &gbuf.p, sizeof(float) * N * ng, "gradient"));
        WP_CK(P, cudaMemsetAsync(gbuf.p, 0, sizeof(float) * N * ng, P->stream));
        for (int i = 0; i < ng; i++) g3[i] = (float *)gbuf.p + i * N;
        WP_TRY(wp_malloc(P, &gphys.p, sizeof(float) * np * nout, "gradient (physical)"));
    }
    if (P->d.kind == PROP_TTI)
        WP_TRY(tti_sweep(P, G, res, (const float *)wbuf.p, (float *)stage.p, grad ? g3 : nullptr));
    else if (P->d.kind == PROP_ACOUSTIC)
        WP_TRY(ac_sweep(P, G, res, (const float *)wbuf.p, (float *)stage.p, grad ? g3[0] : nullptr));
    else
        WP_TRY(el_sweep(P, G, res, (const float *)wbuf.p, (float *)stage.p, grad ? g3 : nullptr));
    if (src_grad) {
        sp_transpose(P, (const float *)stage.p, (float *)out.p, nsrc, nt);
        WP_TRY(copy_out(P, src_grad, (const float *)out.p, (size_t)nt * nsrc));
    }
    if (grad) {
        WP_TRY(ensure_tmp(P, 2));        // fold scratch (free after the sweep)
        if (aniso) tti_axis_to_angles(P, g3 + 3);
        for (int i = 0; i < nout; i++) k_fold(P, g3[i], (float *)gphys.p + i * np, P->tmp[0], P->tmp[1]);
        WP_TRY(copy_out(P, grad, (const float *)gphys.p, np * nout));
    }
    return finish(P);
}

extern "C" int prop_backward(prop_t *P, const float *resid, float *grad, float *src_grad)
{
    WP_TRY(check_handle(P));
    if (!resid) return wp_fail(P, PROP_EINVAL, "resid is NULL");
    int rc = backward_impl(P, resid, grad, src_grad, nullptr);
    free_snaps(P);
    return rc;
}

extern "C" int prop_gradient_aniso(prop_t *P, const float *wavelet, const float *src_xyz, int nsrc,
                                   const float *rec_xyz, int nrec, const float *d_obs, float *grad,
                                   double *misfit)
{
    WP_TRY(check_handle(P));
    if (P->d.kind != PROP_TTI) return wp_fail(P, PROP_EINVAL, "prop_gradient_aniso is for TTI propagators");
    if (!tma_usable(P) && P->d.tti_operator == 1)
        return wp_fail(P, PROP_EINVAL,
                       "prop_gradient_aniso with the staggered-pair operators needs a computational nz that is a "
                       "multiple of 4");
    P->aniso = true;
    const int rc = prop_gradient(P, wavelet, src_xyz, nsrc, rec_xyz, nrec, d_obs, grad, misfit);
    P->aniso = false;
    return rc;
}

extern "C" int prop_stack_image(prop_t *P, const float *image, float *stack, const int *stack_dims,
                                const int *offset, float weight)
{
    WP_TRY(check_handle(P));
    if (!image || !stack || !stack_dims || !offset) return wp_fail(P, PROP_EINVAL, "NULL argument");
    if (!is_dev(stack)) return wp_fail(P, PROP_EINVAL, "stack must be device memory");
    const int n[3] = {P->g.px, P->g.py, P->g.pz};
    for (int a = 0; a < 3; a++)
        if (offset[a] < 0 || stack_dims[a] < 1 || offset[a] + n[a] > stack_dims[a])
            return wp_fail(P, PROP_EINVAL, "window outside the stack");
    DevBuf ibuf;
    const float *img = nullptr;
    WP_TRY(dev_in(P, image, (size_t)n[0] * n[1] * n[2], ibuf, &img));
    k_stack(P, img, stack, stack_dims, offset, weight);
    WP_CK(P, cudaGetLastError());
    return finish(P);
}

extern "C" int prop_trim(prop_t *P)
{
    WP_TRY(check_usable(P));      // launches nothing: the launch count stays
    WP_CK(P, cudaStreamSynchronize(P->stream));
    free_snaps(P);
    for (auto &a : P->st) { cudaFree(a); a = nullptr; }
    for (auto &a : P->ast) { cudaFree(a); a = nullptr; }
    for (auto &a : P->tmp) { cudaFree(a); a = nullptr; }
    P->saved = false;
    P->tmaps.clear();
    if (P->step_graph) {
        cudaGraphExecDestroy(P->step_graph);
        P->step_graph = nullptr;
    }
    return PROP_OK;
}

// device bytes one prop_gradient call allocates on top of what the handle
// already holds (wavefield storage or checkpoints + recompute segment,
// adjoint state, scratch fields, gradient buffers, traces)
static size_t gradient_bytes(const prop_s *P, int nrec)
{
    const size_t N = (size_t)P->g.N, np = (size_t)P->g.px * P->g.py * P->g.pz;
    const int nt = P->d.nt, cf = nfields(P);
    int K = P->d.ckpt_interval;              // without a tail (batches keep none)
    if (K <= 0) K = (int)ceil(sqrt((double)std::max(1, nt - 1)));
    K = std::max(1, std::min(K, std::max(1, nt - 1)));
    const int J = (nt - 1 + K - 1) / K;
    size_t b = 0;
    switch (P->d.snap_mode) {
    case SNAP_FULL_FP32:
        b += (P->d.kind != PROP_ELASTIC ? (size_t)(nt - 1) : (size_t)nt) * snap_fields(P) * N * 4;
        break;
    case SNAP_CKPT_FP32: b += (size_t)J * cf * N * 4; break;
    default: b += (size_t)J * cf * N * 2 + 4 * ((size_t)J * cf + 1024); break;
    }
    if (P->d.snap_mode != SNAP_FULL_FP32)
        b += ((size_t)K + 1) * snap_fields(P) * N * 4;
    for (int i = 0; i < cf; i++) {
        if (!P->ast[i]) b += N * 4;
        if (!P->st[i]) b += N * 4;
    }
    const bool aniso = P->d.kind == PROP_TTI && P->aniso;
    const int ntmp = P->d.kind == PROP_TTI ? (aniso && P->d.tti_operator == 1 ? 20 : aniso || P->d.tti_operator == 1 ? 14 : 8)
                                           : (P->d.kind == PROP_ACOUSTIC ? 0 : 15);
    for (int i = 0; i < ntmp; i++)
        if (!P->tmp[i]) b += N * 4;
    const int ng = P->d.kind == PROP_TTI ? (aniso ? 6 : 1) : (P->d.kind == PROP_ACOUSTIC ? 1 : 3),
              nout = aniso ? 5 : ng;
    b += (N * ng + np * nout) * 4;
    b += (size_t)4 * 4 * nrec * nt;    // traces, staging, observed data, residual
    return b + ((size_t)64 << 20);     // point tables, wavelet, allocator granularity
}

extern "C" size_t prop_gradient_bytes(const prop_t *P, int nrec)
{
    return P ? gradient_bytes(P, std::max(nrec, 0)) : 0;
}

// greedy first-fit of shots, in order, into waves whose bytes sum to at most
// budget; a shot larger than the budget gets a wave of its own
extern "C" int prop_plan_waves(const size_t *bytes, int n, size_t budget, int *wave_of)
{
    if (n < 0 || (n > 0 && (!bytes || !wave_of))) return PROP_EINVAL;
    int w = 0;
    size_t used = 0;
    for (int i = 0; i < n; i++) {
        if (used > 0 && used + bytes[i] > budget) {
            w++;
            used = 0;
        }
        wave_of[i] = w;
        used += bytes[i];
    }
    return n > 0 ? w + 1 : 0;
}

extern "C" int prop_gradient(prop_t *P, const float *wavelet, const float *src_xyz, int nsrc,
                             const float *rec_xyz, int nrec, const float *d_obs, float *grad,
                             double *misfit)
{
    WP_TRY(check_handle(P));
    if (!d_obs || !grad) return wp_fail(P, PROP_EINVAL, "d_obs or grad is NULL");
    const int nt = P->d.nt;
    DevBuf tr, obs;
    WP_TRY(wp_malloc(P, &tr.p, sizeof(float) * (size_t)nrec * nt, "traces"));
    int rc = forward_impl(P, wavelet, src_xyz, nsrc, rec_xyz, nrec, (float *)tr.p, true);
    if (rc) { free_snaps(P); return rc; }
    const float *dobs = nullptr;
    rc = dev_in(P, d_obs, (size_t)nrec * nt, obs, &dobs);
    if (rc) { free_snaps(P); return rc; }
    k_axpy_sq(P, (const float *)tr.p, dobs, (float *)tr.p, (long long)nrec * nt);
    if (misfit) {
        double ss = 0.0;
        rc = k_sumsq(P, (const float *)tr.p, (long long)nrec * nt, &ss);
        if (rc) { free_snaps(P); return rc; }
        *misfit = 0.5 * ss;
    }
    rc = backward_impl(P, (const float *)tr.p, grad, nullptr, nullptr);
    free_snaps(P);
    return rc;
}

// ---------------------------------------------------------------------------
// batched gradients: shots of one wave run concurrently, one host thread and
// one private stream per shot; waves are sized to the free device memory
// ---------------------------------------------------------------------------
#include <thread>

// ---------------------------------------------------------------------------
// Rendezvous of the steps of one wave.  Every shot runs its own
// prop_gradient on its own host thread and stream; the shots' sweeps issue
// their steps in the same order (same nt, storage mode and checkpoint
// interval), so the k-th step of each shot can share one launch per pass.
// A step records an event on the shot's stream and waits for the other
// participants; the last to arrive makes a shared stream wait on all the
// events, launches the batched passes (tile table over all shots; TTI and
// elastic shots of a round in one launch per kind), records `done`, and
// each shot's stream waits on `done` before its next work.  Shots leave the
// group when their gradient returns, so participants with other step
// sequences never wait for each other; steps that cannot share a launch
// (different step kinds of one propagator in a round) run one by one.
// ---------------------------------------------------------------------------
struct RdvReq {
    int kind;                 // 1 TTI step, 2 elastic step
    TtiBatchReq t;
    ElBatchReq e;
};

struct StepRendezvous {
    std::mutex mu;
    std::condition_variable cv;
    int active = 0, arrived = 0;
    unsigned long long gen = 0;
    std::vector<RdvReq> req;
    std::vector<char> present;
    std::vector<cudaEvent_t> ev;
    std::vector<int> result;      // 0 launched, 1 launch alone, < 0 error
    cudaStream_t cs = nullptr;
    cudaEvent_t done[2] = {};
    TtiBatch *tb = nullptr, *eb = nullptr;   // tables of the TTI and of the elastic shots
    std::string err;
    long long batched = 0, alone = 0;

    ~StepRendezvous()
    {
        if (cs) cudaStreamSynchronize(cs);
        tti_batch_free(tb);
        tti_batch_free(eb);
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        for (auto e : done)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    }
    int init(int n)
    {
        req.resize(n);
        present.assign(n, 0);
        ev.assign(n, nullptr);
        result.assign(n, 0);
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PROP_ECUDA;
        for (auto &e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PROP_ECUDA;
        for (auto &e : done)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PROP_ECUDA;
        tb = tti_batch_new();
        eb = tti_batch_new();
        return PROP_OK;
    }
    // with the lock held, by the last participant to arrive: one shared
    // launch per kind of step present in the round
    void launch_all()
    {
        std::vector<TtiBatchReq> rt;
        std::vector<ElBatchReq> re;
        std::vector<int> wt, we;
        for (size_t i = 0; i < req.size(); i++)
            if (present[i]) {
                cudaStreamWaitEvent(cs, ev[i], 0);
                if (req[i].kind == 1) {
                    rt.push_back(req[i].t);
                    wt.push_back((int)i);
                } else {
                    re.push_back(req[i].e);
                    we.push_back((int)i);
                }
            }
        bool any = false;
        auto settle = [&](int rc, const std::vector<int> &who) {
            if (who.empty()) return;
            if (rc == PROP_OK) {
                batched++;
                any = true;
            } else if (rc == 1) {
                alone++;
            }
            for (int i : who) result[i] = rc;
        };
        settle(rt.empty() ? PROP_OK : tti_batch_step(tb, rt.data(), (int)rt.size(), cs, &err), wt);
        settle(re.empty() ? PROP_OK : el_batch_step(eb, re.data(), (int)re.size(), cs, &err), we);
        if (any && cudaEventRecord(done[gen & 1], cs) != cudaSuccess) {
            err = "batched step: event record failed";
            for (size_t i = 0; i < req.size(); i++)
                if (present[i] && result[i] == PROP_OK) result[i] = PROP_ECUDA;
        }
        for (size_t i = 0; i < req.size(); i++) present[i] = 0;
        arrived = 0;
        gen++;
        cv.notify_all();
    }
    void leave()
    {
        std::lock_guard<std::mutex> lk(mu);
        active--;
        if (active > 0 && arrived == active) launch_all();
    }
    // one shot's step: deposit, wait for the round, then order the shot's
    // stream after the shared launch (0), or tell it to launch alone (1)
    int meet(prop_s *P, const RdvReq &r, cudaEvent_t *d)
    {
        const int i = P->rdv_idx;
        std::unique_lock<std::mutex> lk(mu);
        const cudaError_t e = cudaEventRecord(ev[i], P->stream);
        if (e != cudaSuccess) return wp_cuda(P, e, "cudaEventRecord (batched step)");
        req[i] = r;
        present[i] = 1;
        const unsigned long long my = gen;
        if (++arrived == active) launch_all();
        else cv.wait(lk, [&] { return gen != my; });
        *d = done[my & 1];
        if (result[i] < 0) return wp_fail(P, result[i], err);
        return result[i];
    }
};

int rdv_tti_step(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r, float *grad)
{
    StepRendezvous *R = P->rdv;
    RdvReq r{};
    r.kind = 1;
    r.t = TtiBatchReq{P, {S[0], S[1], S[2], S[3]}, adjoint, img_p, img_r, grad};
    cudaEvent_t d = nullptr;
    const int res = R->meet(P, r, &d);
    if (res < 0) return res;
    if (res == 1) {                 // could not share the launch: this shot alone
        P->rdv = nullptr;
        const int rc = tti_launch_step(P, S, adjoint, img_p, img_r, grad);
        P->rdv = R;
        return rc;
    }
    WP_CK(P, cudaStreamWaitEvent(P->stream, d, 0));
    return PROP_OK;
}

int rdv_el_step(prop_s *P, const ElBatchReq &e)
{
    StepRendezvous *R = P->rdv;
    RdvReq r{};
    r.kind = 2;
    r.e = e;
    cudaEvent_t d = nullptr;
    const int res = R->meet(P, r, &d);
    if (res < 0) return res;
    if (res == 1) {
        P->rdv = nullptr;
        int rc;
        if (e.mode == 1) rc = el_launch_adj_grad(P, e.S, e.xk, e.xk1, e.g);
        else if (e.sign < 0.f) rc = el_step_adjoint_u(P, e.S);
        else rc = el_launch_step(P, e.S, false);
        P->rdv = R;
        return rc;
    }
    WP_CK(P, cudaStreamWaitEvent(P->stream, d, 0));
    return PROP_OK;
}

// ---------------------------------------------------------------------------
// Forward modelling of many TTI (or many elastic) shots in lockstep: per
// time step the receivers of every shot are sampled, one tile-table launch
// of each pass advances every shot, and the sources are injected.  The TTI
// state buffers rotate with period 2 (the elastic state is updated in
// place), so two steps are captured once into a CUDA graph (the sparse
// kernels read the time index from device memory and a one-thread kernel
// advances it) and the graph is replayed nt/2 times.
// ---------------------------------------------------------------------------
static int forward_batch_one_by_one(prop_t *const *shots, int n, const float *const *wavelet,
                                    const float *const *src_xyz, const int *nsrc, const float *const *rec_xyz,
                                    const int *nrec, float *const *traces)
{
    for (int i = 0; i < n; i++) {
        const int rc = prop_forward(shots[i], wavelet[i], src_xyz[i], nsrc[i], rec_xyz[i], nrec[i], traces[i]);
        if (rc) {
            tl_err = "shot " + std::to_string(i) + ": " + prop_last_error(shots[i]);
            return rc;
        }
    }
    return PROP_OK;
}

extern "C" int prop_forward_batch(prop_t *const *shots, int n, const float *const *wavelet,
                                  const float *const *src_xyz, const int *nsrc, const float *const *rec_xyz,
                                  const int *nrec, float *const *traces)
{
    if (n < 0) return wp_fail(nullptr, PROP_EINVAL, "nshots < 0");
    if (n == 0) return PROP_OK;
    if (!shots || !wavelet || !src_xyz || !nsrc || !rec_xyz || !nrec || !traces)
        return wp_fail(nullptr, PROP_EINVAL, "NULL array argument");
    for (int i = 0; i < n; i++) {
        if (!shots[i]) return wp_fail(nullptr, PROP_EINVAL, "shot handle " + std::to_string(i) + " is NULL");
        for (int j = 0; j < i; j++)
            if (shots[j] == shots[i])
                return wp_fail(nullptr, PROP_EINVAL, "shot handle " + std::to_string(i) + " repeats an earlier one");
        if (!wavelet[i] || !src_xyz[i] || !rec_xyz[i] || !traces[i] || nsrc[i] < 1 || nrec[i] < 1)
            return wp_fail(nullptr, PROP_EINVAL, "shot " + std::to_string(i) + ": missing wavelet, geometry or output");
    }
    // lockstep needs TTI shots (or elastic shots) on the TMA-fed passes with
    // one space order and nt
    const bool el = el_batchable(shots[0]);
    bool lock = true;
    for (int i = 0; i < n && lock; i++)
        lock = (el ? el_batchable(shots[i]) : tti_batchable(shots[i])) && shots[i]->M == shots[0]->M &&
               shots[i]->d.nt == shots[0]->d.nt && !shots[i]->broken;
    // as for gradients, lockstep pays on small windows: elastic, 32 shots of
    // about 1 M points 168.5k against 153.0k shots/h; of 30-110 M points
    // 7,269 against 7,976 (the windows fill the GPU one at a time).
    // WAVEPROP_LOCKSTEP=1 forces it for any size, =0 disables it.
    const char *ls = getenv("WAVEPROP_LOCKSTEP");
    double pts = 0.0;
    for (int i = 0; i < n; i++) pts += (double)shots[i]->g.N;
    if (ls && !strcmp(ls, "0")) lock = false;
    else if (!(ls && !strcmp(ls, "1")) && pts / n > 16.0e6) lock = false;
    const char *bl = getenv("WAVEPROP_BATCH_LAUNCH");
    if (!lock || n < 2 || (bl && !strcmp(bl, "0")))
        return forward_batch_one_by_one(shots, n, wavelet, src_xyz, nsrc, rec_xyz, nrec, traces);

    prop_s *P0 = shots[0];
    const int nt = P0->d.nt;
    // every shot's work runs on one private stream (capturable, unlike the
    // legacy default stream), after what each handle had queued on its own
    // stream; each handle's stream waits for the batch at the end
    struct OwnStream {
        cudaStream_t s = nullptr;
        ~OwnStream()
        {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        }
    } bs;
    WP_CK(P0, cudaStreamCreateWithFlags(&bs.s, cudaStreamNonBlocking));
    const cudaStream_t st = bs.s;
    std::vector<cudaStream_t> own(n);
    struct Restore {
        prop_t *const *sh;
        std::vector<cudaStream_t> *own;
        int n;
        ~Restore()
        {
            for (int i = 0; i < n; i++) sh[i]->stream = (*own)[i];
        }
    } restore{shots, &own, 0};
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        WP_TRY(check_handle(P));
        own[i] = P->stream;
        if (P->stream != st) {
            cudaEvent_t e;
            WP_CK(P, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            cudaEventRecord(e, P->stream);
            cudaStreamWaitEvent(st, e, 0);
            cudaEventDestroy(e);
        }
        P->stream = st;
        restore.n = i + 1;
        WP_TRY(ensure_work(P));
    }
    std::vector<Geometry> G(n);
    std::vector<DevBuf> wb(n), stage(n), tr(n);
    std::vector<const float *> wav(n);
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        WP_TRY(build_geometry(P, G[i], src_xyz[i], nsrc[i], rec_xyz[i], nrec[i]));
        WP_TRY(dev_in(P, wavelet[i], (size_t)nsrc[i] * nt, wb[i], &wav[i]));
        WP_TRY(wp_malloc(P, &stage[i].p, sizeof(float) * (size_t)nt * nrec[i], "trace staging"));
        WP_TRY(wp_malloc(P, &tr[i].p, sizeof(float) * (size_t)nt * nrec[i], "traces"));
        WP_TRY(zero_fields(P, P->st, nfields(P)));
    }
    DevBuf tbuf;
    WP_TRY(wp_malloc(P0, &tbuf.p, sizeof(int), "time index"));
    int *tdev = (int *)tbuf.p;
    WP_CK(P0, cudaMemsetAsync(tdev, 0, sizeof(int), st));
    // TTI: the two buffer arrangements of a step, (p, r, p_prev, r_prev) and
    // the rotated one; elastic: one (the state is updated in place)
    std::unique_ptr<TtiBatch, void (*)(TtiBatch *)> tb(tti_batch_new(), tti_batch_free);
    for (int c = 0; c < (el ? 1 : 2); c++) {
        std::string err;
        int rc;
        if (el) {
            std::vector<ElBatchReq> req(n);
            for (int i = 0; i < n; i++) {
                req[i] = ElBatchReq{shots[i], {}, 0, 1.f, {}, {}, {}};
                for (int k = 0; k < 9; k++) req[i].S[k] = shots[i]->st[k];
            }
            rc = el_batch_fix(tb.get(), req.data(), n, 0, st, &err);
        } else {
            std::vector<TtiBatchReq> req(n);
            for (int i = 0; i < n; i++) {
                float *const *q = shots[i]->st;
                req[i] = c == 0 ? TtiBatchReq{shots[i], {q[0], q[1], q[2], q[3]}, false, nullptr, nullptr, nullptr}
                                : TtiBatchReq{shots[i], {q[2], q[3], q[0], q[1]}, false, nullptr, nullptr, nullptr};
            }
            rc = tti_batch_fix(tb.get(), req.data(), n, c, st, &err);
        }
        if (rc == 1) return forward_batch_one_by_one(shots, n, wavelet, src_xyz, nsrc, rec_xyz, nrec, traces);
        if (rc) return wp_fail(P0, rc, err);
    }
    // one step in arrangement c: record d^n from u^n, advance every shot,
    // inject q^n into the new level, t += 1 (elastic: receivers record the
    // trace of the stress, the source enters tau_xx, tau_yy, tau_zz)
    auto step = [&](int c) -> int {
        for (int i = 0; i < n; i++) {
            prop_s *P = shots[i];
            float *const *q = P->st;
            if (el) sp_record(P, &G[i].R, q[3], q[4], q[5], 1.f, (float *)stage[i].p, tdev);
            else sp_record(P, &G[i].R, c == 0 ? q[0] : q[2], nullptr, nullptr, 1.f, (float *)stage[i].p, tdev);
        }
        if ((el ? el_batch_launch_fixed(tb.get(), 0, st) : tti_batch_launch_fixed(tb.get(), c, st)) != PROP_OK)
            return wp_fail(P0, PROP_ECUDA, "batched step launch failed");
        for (int i = 0; i < n; i++) {
            prop_s *P = shots[i];
            float *const *q = P->st;
            if (el) {
                sp_inject(P, &G[i].S, wav[i], nt, 0, P->g.dt, 0, q[3], q[4], q[5], nullptr, nullptr, tdev);
            } else {
                float *pn = c == 0 ? q[2] : q[0], *rn = c == 0 ? q[3] : q[1];
                sp_inject(P, &G[i].S, wav[i], nt, 0, P->g.dt * P->g.dt, 1, pn, rn, nullptr, nullptr, nullptr,
                          tdev);
            }
            P->kern_launches += 1;      // the shared pass launches, counted once per shot
        }
        k_tick(P0, tdev, 1);
        return PROP_OK;
    };
    const char *ge = getenv("WAVEPROP_GRAPHS");
    const bool graphs = !(ge && !strcmp(ge, "0")) && nt >= 4;
    int done = 0;
    if (graphs) {
        cudaGraph_t gr = nullptr;
        cudaGraphExec_t ex = nullptr;
        std::vector<long long> before(n);
        for (int i = 0; i < n; i++) before[i] = shots[i]->kern_launches;
        WP_CK(P0, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const int r0 = step(0), r1 = r0 ? r0 : step(1);
        const cudaError_t ec = cudaStreamEndCapture(st, &gr);
        if (r1 || ec != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            if (r1) return r1;
            return wp_cuda(P0, ec, "capture of the batched steps");
        }
        const cudaError_t ei = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        WP_CK(P0, ei);
        for (; done + 2 <= nt; done += 2) {
            const cudaError_t el = cudaGraphLaunch(ex, st);
            if (el != cudaSuccess) {
                cudaGraphExecDestroy(ex);
                return wp_cuda(P0, el, "cudaGraphLaunch (batched steps)");
            }
        }
        WP_CK(P0, cudaStreamSynchronize(st));
        cudaGraphExecDestroy(ex);
        // the capture counted the launches of one replay
        for (int i = 0; i < n; i++)
            shots[i]->kern_launches += (shots[i]->kern_launches - before[i]) * (done / 2 - 1);
    }
    for (; done < nt; done++) WP_TRY(step(done & 1));
    // the final state in st[] order (TTI: odd nt leaves the rotated arrangement)
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        if ((nt & 1) && !el) {
            std::swap(P->st[0], P->st[2]);
            std::swap(P->st[1], P->st[3]);
        }
        sp_transpose(P, (const float *)stage[i].p, (float *)tr[i].p, nrec[i], nt);
        WP_TRY(copy_out(P, traces[i], (const float *)tr[i].p, (size_t)nt * nrec[i]));
    }
    int first = PROP_OK;
    for (int i = 0; i < n; i++) {
        const int rc = finish(shots[i]);
        if (rc && !first) {
            first = rc;
            tl_err = "shot " + std::to_string(i) + ": " + prop_last_error(shots[i]);
        }
    }
    // each handle's own stream continues after the batch
    for (int i = 0; i < n; i++)
        if (own[i] != st) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, st);
                cudaStreamWaitEvent(own[i], e, 0);
                cudaEventDestroy(e);
            }
        }
    return first;
}

// shared step launches of the calling thread's last prop_gradient_batch
// call: rounds launched together (rendezvous rounds and lockstep steps),
// rounds whose steps had to be launched one by one
static thread_local long long batch_stats[2] = {0, 0};
extern "C" int prop_batch_stats(long long *shared, long long *alone)
{
    if (shared) *shared = batch_stats[0];
    if (alone) *alone = batch_stats[1];
    return PROP_OK;
}

// ---------------------------------------------------------------------------
// Gradients of a wave of TTI shots in lockstep (same space order, nt and
// checkpoint schedule, centred operators on the TMA-fed passes, checkpointed
// storage): one host thread drives every shot through the same sweep.
//   forward:  per step, the receivers of every shot are sampled, one
//             tile-table launch of each pass advances every shot and the
//             sources are injected; a checkpoint is saved at the start of
//             each segment of K steps;
//   adjoint:  per segment (last first), every shot's checkpoint is loaded,
//             K steps are recomputed into the segment buffers, then K
//             transposed steps with imaging run (one launch of each pass
//             for every shot) with the residual injected after each.
// The time index lives in device memory, the per-shot tables of every step
// configuration (two forward arrangements; the transposed step for each
// position in the segment and each arrangement of the adjoint state) are
// fixed device tables, so the K steps of a forward segment and the 2K steps
// of an adjoint segment are each captured once as a CUDA graph and replayed
// for every full segment; checkpoint saves and loads, partial segments and
// WAVEPROP_GRAPHS=0 launch directly.  Each shot's operations are those of its
// own prop_gradient, in the same order, so the results are the same bits.
// Returns 1 (nothing done) if the wave does not qualify.
// ---------------------------------------------------------------------------

static bool lockstep_ok(prop_t *const *sh, int n)
{
    if (n < 2) return false;
    const prop_s *P0 = sh[0];
    const bool el = el_batchable(P0);
    for (int i = 0; i < n; i++) {
        const prop_s *P = sh[i];
        if (!(el ? el_batchable(P) : tti_batchable(P)) || P->broken || P->aniso || P->M != P0->M ||
            P->d.nt != P0->d.nt ||
            P->d.snap_mode == SNAP_FULL_FP32 || P->d.snap_mode != P0->d.snap_mode ||
            P->d.ckpt_interval != P0->d.ckpt_interval)
            return false;
    }
    // the lockstep driver pays where the rounds are paced by the host (small
    // windows: 32 windows of about 1 M points, 0.99 s against 1.01 s for
    // one thread per shot); on windows of tens of millions of points the
    // per-thread rendezvous measured 4 % faster (6.26 s against 6.51 s for 8
    // shots of 30-110 M points).  WAVEPROP_LOCKSTEP=1 forces it, =0 disables it.
    const char *e = getenv("WAVEPROP_LOCKSTEP");
    if (e && !strcmp(e, "0")) return false;
    if (e && !strcmp(e, "1")) return true;
    double pts = 0.0;
    for (int i = 0; i < n; i++) pts += (double)sh[i]->g.N;
    return pts / n <= 16.0e6;
}

static int gradient_lockstep(prop_t *const *shots, int n, const float *const *wavelet,
                             const float *const *src_xyz, const int *nsrc, const float *const *rec_xyz,
                             const int *nrec, const float *const *d_obs, float *const *grad, double *mis)
{
    prop_s *P0 = shots[0];
    const int nt = P0->d.nt;
    struct OwnStream {
        cudaStream_t s = nullptr;
        ~OwnStream()
        {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        }
    } bs;
    WP_CK(P0, cudaStreamCreateWithFlags(&bs.s, cudaStreamNonBlocking));
    const cudaStream_t st = bs.s;
    // WAVEPROP_BATCH_VERBOSE=1: wall time of each phase on stderr (the
    // stream is synchronised at the phase ends)
    const char *vb = getenv("WAVEPROP_BATCH_VERBOSE");
    const bool verbose = vb && !strcmp(vb, "1");
    auto tnow = [] { return std::chrono::steady_clock::now(); };
    auto tlast = tnow();
    auto phase = [&](const char *name) {
        if (!verbose) return;
        cudaStreamSynchronize(st);
        const auto t = tnow();
        fprintf(stderr, "lockstep %d shots: %-10s %9.3f ms\n", n, name,
                std::chrono::duration<double, std::milli>(t - tlast).count());
        tlast = t;
    };
    std::vector<cudaStream_t> own(n);
    struct Restore {            // streams and the tail switch of every shot
        prop_t *const *sh;
        std::vector<cudaStream_t> *own;
        int n;
        ~Restore()
        {
            for (int i = 0; i < n; i++) {
                sh[i]->stream = (*own)[i];
                sh[i]->no_tail = false;
                free_snaps(sh[i]);
            }
        }
    } restore{shots, &own, 0};
    // a wave whose setup fails (a bad argument of one shot, or the memory of
    // the whole wave) runs shot by shot instead, so that each call reports
    // its own error
    for (int i = 0; i < n; i++)
        if (!d_obs[i] || !grad[i] || !wavelet[i] || !src_xyz[i] || !rec_xyz[i] || nsrc[i] < 1 || nrec[i] < 1)
            return 1;
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        if (check_handle(P) != PROP_OK) return 1;
        own[i] = P->stream;
        cudaEvent_t e;
        WP_CK(P, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, P->stream);
        cudaStreamWaitEvent(st, e, 0);
        cudaEventDestroy(e);
        P->stream = st;
        P->no_tail = true;
        restore.n = i + 1;
        if (ensure_work(P) != PROP_OK || ensure_ast(P) != PROP_OK) return 1;
    }
    // every allocation before the first capture
    std::vector<Geometry> G(n);
    std::vector<DevBuf> wb(n), ob(n), stage(n), tr(n), gb(n), gp(n);
    std::vector<const float *> wav(n), obs(n);
    auto setup = [&](int i) -> int {
        prop_s *P = shots[i];
        const size_t N = (size_t)P->g.N, np = (size_t)P->g.px * P->g.py * P->g.pz;
        WP_TRY(build_geometry(P, G[i], src_xyz[i], nsrc[i], rec_xyz[i], nrec[i]));
        WP_TRY(dev_in(P, wavelet[i], (size_t)nsrc[i] * nt, wb[i], &wav[i]));
        WP_TRY(dev_in(P, d_obs[i], (size_t)nrec[i] * nt, ob[i], &obs[i]));
        WP_TRY(wp_malloc(P, &stage[i].p, sizeof(float) * (size_t)nt * nrec[i], "trace staging"));
        WP_TRY(wp_malloc(P, &tr[i].p, sizeof(float) * (size_t)nt * nrec[i], "traces"));
        WP_TRY(wp_malloc(P, &gb[i].p, sizeof(float) * N, "gradient"));
        WP_TRY(wp_malloc(P, &gp[i].p, sizeof(float) * np, "gradient (physical)"));
        WP_CK(P, cudaMemsetAsync(gb[i].p, 0, sizeof(float) * N, st));
        WP_TRY(alloc_saves(P));
        WP_TRY(zero_fields(P, P->st, 4));
        WP_TRY(zero_fields(P, P->ast, 4));
        WP_TRY(zero_fields(P, P->tmp + 6, 2));     // zeta = C lam of the zero state
        return PROP_OK;
    };
    phase("handles");
    for (int i = 0; i < n; i++)
        if (setup(i) != PROP_OK) {
            cudaStreamSynchronize(st);
            return 1;
        }
    phase("setup");
    const int K = ckpt_K(P0), J = ckpt_J(P0), span = ckpt_span(P0);
    for (int i = 1; i < n; i++)
        if (ckpt_K(shots[i]) != K || ckpt_J(shots[i]) != J || ckpt_span(shots[i]) != span) return 1;
    DevBuf tbuf;
    WP_TRY(wp_malloc(P0, &tbuf.p, sizeof(int), "time index"));
    int *tdev = (int *)tbuf.p;
    // fixed tables: slots 0, 1 the forward arrangements of the state (the
    // recomputation starts from the same arrangement in every segment);
    // slot 2 + 2p + q the transposed step with imaging at segment position p
    // (forward level n0 + p + 1 in segment buffer p) in adjoint arrangement q
    std::unique_ptr<TtiBatch, void (*)(TtiBatch *)> tb(tti_batch_new(), tti_batch_free);
    std::vector<TtiBatchReq> req(n);
    std::string err;
    for (int c = 0; c < 2; c++) {
        for (int i = 0; i < n; i++) {
            float *const *q = shots[i]->st;
            req[i] = c == 0 ? TtiBatchReq{shots[i], {q[0], q[1], q[2], q[3]}, false, nullptr, nullptr, nullptr}
                            : TtiBatchReq{shots[i], {q[2], q[3], q[0], q[1]}, false, nullptr, nullptr, nullptr};
        }
        const int rc = tti_batch_fix(tb.get(), req.data(), n, c, st, &err);
        if (rc) return rc == 1 ? 1 : wp_fail(P0, rc, err);
    }
    for (int pos = 0; pos < K; pos++)
        for (int qa = 0; qa < 2; qa++) {
            for (int i = 0; i < n; i++) {
                prop_s *P = shots[i];
                float *const *a = P->ast;
                const float *u = P->seg + (size_t)pos * 2 * (size_t)P->g.N;
                req[i] = qa == 0 ? TtiBatchReq{P, {a[0], a[1], a[2], a[3]}, true, u, u + P->g.N, (float *)gb[i].p}
                                 : TtiBatchReq{P, {a[2], a[3], a[0], a[1]}, true, u, u + P->g.N, (float *)gb[i].p};
            }
            const int rc = tti_batch_fix(tb.get(), req.data(), n, 2 + 2 * pos + qa, st, &err);
            if (rc) return rc == 1 ? 1 : wp_fail(P0, rc, err);
        }
    phase("tables");
    auto launch = [&](int slot) -> int {
        if (tti_batch_launch_fixed(tb.get(), slot, st) != PROP_OK)
            return wp_fail(P0, PROP_ECUDA, "batched TTI step launch failed");
        for (int i = 0; i < n; i++) shots[i]->kern_launches += 1;
        batch_stats[0]++;
        return PROP_OK;
    };
    // The per-shot kernels of a step (receiver sampling, injection, segment
    // copies) are small: shot i runs them on worker stream i % W, forked from
    // and joined back into the shared stream, so that different shots' run
    // side by side (parallel branches when captured).
    constexpr int W = 8;
    struct Workers {
        cudaStream_t s[W] = {};
        cudaEvent_t fork = nullptr, join[W] = {};
        ~Workers()
        {
            for (auto x : s)
                if (x) cudaStreamDestroy(x);
            if (fork) cudaEventDestroy(fork);
            for (auto e : join)
                if (e) cudaEventDestroy(e);
        }
    } wk;
    const int nwk = std::min(W, n);
    WP_CK(P0, cudaEventCreateWithFlags(&wk.fork, cudaEventDisableTiming));
    for (int w = 0; w < nwk; w++) {
        WP_CK(P0, cudaStreamCreateWithFlags(&wk.s[w], cudaStreamNonBlocking));
        WP_CK(P0, cudaEventCreateWithFlags(&wk.join[w], cudaEventDisableTiming));
    }
    auto per_shot = [&](const std::function<int(int)> &fn) -> int {
        WP_CK(P0, cudaEventRecord(wk.fork, st));
        for (int w = 0; w < nwk; w++) WP_CK(P0, cudaStreamWaitEvent(wk.s[w], wk.fork, 0));
        int rc = PROP_OK;
        for (int i = 0; i < n && !rc; i++) {
            shots[i]->stream = wk.s[i % nwk];
            rc = fn(i);
            shots[i]->stream = st;
        }
        for (int w = 0; w < nwk; w++) {
            WP_CK(P0, cudaEventRecord(wk.join[w], wk.s[w]));
            WP_CK(P0, cudaStreamWaitEvent(st, wk.join[w], 0));
        }
        return rc;
    };
    // forward step in arrangement c: record d^t, step, inject q^t (and, in
    // the recomputation, copy the new level into segment buffer pos), t += 1
    auto fwd = [&](int c, bool record, int pos) -> int {
        if (record)
            WP_TRY(per_shot([&](int i) -> int {
                float *const *q = shots[i]->st;
                sp_record(shots[i], &G[i].R, c == 0 ? q[0] : q[2], nullptr, nullptr, 1.f, (float *)stage[i].p,
                          tdev);
                return PROP_OK;
            }));
        WP_TRY(launch(c));
        WP_TRY(per_shot([&](int i) -> int {
            prop_s *P = shots[i];
            float *const *q = P->st;
            float *pn = c == 0 ? q[2] : q[0], *rn = c == 0 ? q[3] : q[1];
            sp_inject(P, &G[i].S, wav[i], nt, 0, P->g.dt * P->g.dt, 1, pn, rn, nullptr, nullptr, nullptr, tdev);
            if (pos >= 0) {
                const size_t N = (size_t)P->g.N;
                float *d = P->seg + (size_t)pos * 2 * N;
                WP_CK(P, cudaMemcpyAsync(d, pn, N * 4, cudaMemcpyDeviceToDevice, P->stream));
                WP_CK(P, cudaMemcpyAsync(d + N, rn, N * 4, cudaMemcpyDeviceToDevice, P->stream));
            }
            return PROP_OK;
        }));
        k_tick(P0, tdev, 1);
        return PROP_OK;
    };
    // recomputed forward step at segment position pos
    auto recompute = [&](int pos) -> int { return fwd(pos & 1, false, pos); };
    // transposed step k = t with imaging at position pos, adjoint
    // arrangement qa; residual r^k into the new level; t -= 1
    auto adj = [&](int pos, int qa) -> int {
        WP_TRY(launch(2 + 2 * pos + qa));
        WP_TRY(per_shot([&](int i) -> int {
            prop_s *P = shots[i];
            float *const *a = P->ast;
            const float *u = P->seg + (size_t)pos * 2 * (size_t)P->g.N;
            sp_inject(P, &G[i].R, (const float *)tr[i].p, nt, 0, 1.f, 3, qa == 0 ? a[2] : a[0], P->tmp[6],
                      P->tmp[7], u, (float *)gb[i].p, tdev);
            return PROP_OK;
        }));
        k_tick(P0, tdev, -1);
        return PROP_OK;
    };
    const char *ge = getenv("WAVEPROP_GRAPHS");
    const bool graphs = !(ge && !strcmp(ge, "0"));
    struct Graphs {             // destroyed only after the stream's work (error paths too)
        cudaStream_t st;
        cudaGraphExec_t g[4] = {};
        ~Graphs()
        {
            cudaStreamSynchronize(st);
            for (auto e : g)
                if (e) cudaGraphExecDestroy(e);
        }
    } gx{st};
    std::vector<long long> held[4];     // launches each graph holds, per shot
    // run body() directly, or from graph `id` (captured on first use)
    auto run = [&](int id, const std::function<int()> &body) -> int {
        if (!graphs) return body();
        if (!gx.g[id]) {
            std::vector<long long> before(n);
            for (int i = 0; i < n; i++) before[i] = shots[i]->kern_launches;
            cudaGraph_t gr = nullptr;
            WP_CK(P0, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int rb = body();
            const cudaError_t ec = cudaStreamEndCapture(st, &gr);
            if (rb || ec != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                cudaGetLastError();
                return rb ? rb : wp_cuda(P0, ec, "capture of the lockstep segment");
            }
            const cudaError_t ei = cudaGraphInstantiate(&gx.g[id], gr, 0);
            cudaGraphDestroy(gr);
            WP_CK(P0, ei);
            held[id].resize(n);
            for (int i = 0; i < n; i++) held[id][i] = shots[i]->kern_launches - before[i];
        } else {
            for (int i = 0; i < n; i++) shots[i]->kern_launches += held[id][i];
        }
        WP_CK(P0, cudaGraphLaunch(gx.g[id], st));
        return PROP_OK;
    };
    // ---- forward sweep with checkpoints ----
    k_set_int(P0, tdev, 0);
    for (int j = 0; j < J; j++) {
        const int n0 = j * K, n1 = j + 1 < J ? n0 + K : nt;     // steps n0 .. n1-1
        const int c0 = n0 & 1;
        WP_TRY(per_shot([&](int i) -> int {
            float *const *q = shots[i]->st;
            float *s4[4] = {q[0], q[1], q[2], q[3]};
            if (c0) s4[0] = q[2], s4[1] = q[3], s4[2] = q[0], s4[3] = q[1];
            return save_checkpoint(shots[i], j, s4);
        }));
        auto body = [&]() -> int {
            for (int t = n0; t < n1; t++) WP_TRY(fwd(t & 1, true, -1));
            return PROP_OK;
        };
        if (n1 - n0 == K) WP_TRY(run(c0, body));
        else WP_TRY(body());
    }
    phase("forward");
    // ---- residuals and misfits ----
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        const long long m = (long long)nrec[i] * nt;
        sp_transpose(P, (const float *)stage[i].p, (float *)tr[i].p, nrec[i], nt);
        k_axpy_sq(P, (const float *)tr[i].p, obs[i], (float *)tr[i].p, m);
        double ss = 0.0;
        WP_TRY(k_sumsq(P, (const float *)tr[i].p, m, &ss));
        mis[i] = 0.5 * ss;
    }
    phase("misfit");
    // ---- adjoint sweep over the segments, last first ----
    int qa = 0;                    // arrangement of the adjoint state
    for (int j = J - 1; j >= 0; j--) {
        const int n0 = j * K, E = std::min(n0 + K, span), len = E - n0;
        WP_TRY(per_shot([&](int i) -> int { return load_checkpoint(shots[i], j, shots[i]->st); }));
        k_set_int(P0, tdev, n0);
        const int q0 = qa;
        auto body = [&]() -> int {
            for (int pos = 0; pos < len; pos++) WP_TRY(recompute(pos));
            for (int k = E, q = q0; k >= n0 + 1; k--, q ^= 1) WP_TRY(adj(k - n0 - 1, q));
            return PROP_OK;
        };
        if (len == K) WP_TRY(run(2 + q0, body));
        else WP_TRY(body());
        qa = (qa + len) & 1;
    }
    phase("adjoint");
    // ---- gradients on the physical grid ----
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        const size_t np = (size_t)P->g.px * P->g.py * P->g.pz;
        k_fold(P, (const float *)gb[i].p, (float *)gp[i].p, P->tmp[0], P->tmp[1]);
        WP_TRY(copy_out(P, grad[i], (const float *)gp[i].p, np));
    }
    int first = PROP_OK;
    for (int i = 0; i < n; i++) {
        const int rc = finish(shots[i]);
        if (rc && !first) {
            first = rc;
            tl_err = "shot " + std::to_string(i) + ": " + prop_last_error(shots[i]);
        }
    }
    phase("gradients");
    for (int i = 0; i < n; i++) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(e, st);
            cudaStreamWaitEvent(own[i], e, 0);
            cudaEventDestroy(e);
        }
    }
    return first;
}

// ---------------------------------------------------------------------------
// Gradients of a wave of elastic shots in lockstep (same space order, nt and
// checkpoint schedule, TMA-fed passes, checkpointed storage): as for TTI,
// one host thread; the state and the adjoint state are updated in place, so
// one fixed table serves every forward step and one per segment position
// the transposed step with imaging (its three passes; the pointwise kernels
// before and after it run per shot).  Full segments (K recomputed steps and
// K transposed steps) are captured once as a CUDA graph and replayed.
// Each shot's operations are those of its own prop_gradient, in the same
// order, so the results are the same bits.  Returns 1 (nothing done) if the
// wave does not qualify.
// ---------------------------------------------------------------------------
static int el_gradient_lockstep(prop_t *const *shots, int n, const float *const *wavelet,
                                const float *const *src_xyz, const int *nsrc, const float *const *rec_xyz,
                                const int *nrec, const float *const *d_obs, float *const *grad, double *mis)
{
    prop_s *P0 = shots[0];
    const int nt = P0->d.nt;
    struct OwnStream {
        cudaStream_t s = nullptr;
        ~OwnStream()
        {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        }
    } bs;
    WP_CK(P0, cudaStreamCreateWithFlags(&bs.s, cudaStreamNonBlocking));
    const cudaStream_t st = bs.s;
    std::vector<cudaStream_t> own(n);
    struct Restore {
        prop_t *const *sh;
        std::vector<cudaStream_t> *own;
        int n;
        ~Restore()
        {
            for (int i = 0; i < n; i++) {
                sh[i]->stream = (*own)[i];
                free_snaps(sh[i]);
            }
        }
    } restore{shots, &own, 0};
    for (int i = 0; i < n; i++)
        if (!d_obs[i] || !grad[i] || !wavelet[i] || !src_xyz[i] || !rec_xyz[i] || nsrc[i] < 1 || nrec[i] < 1)
            return 1;
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        if (check_handle(P) != PROP_OK) return 1;
        own[i] = P->stream;
        cudaEvent_t e;
        WP_CK(P, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, P->stream);
        cudaStreamWaitEvent(st, e, 0);
        cudaEventDestroy(e);
        P->stream = st;
        restore.n = i + 1;
        if (ensure_work(P) != PROP_OK || ensure_ast(P) != PROP_OK || ensure_tmp(P, 15) != PROP_OK) return 1;
    }
    std::vector<Geometry> G(n);
    std::vector<DevBuf> wb(n), ob(n), stage(n), tr(n), gb(n), gp(n);
    std::vector<const float *> wav(n), obs(n);
    auto setup = [&](int i) -> int {
        prop_s *P = shots[i];
        const size_t N = (size_t)P->g.N, np = (size_t)P->g.px * P->g.py * P->g.pz;
        WP_TRY(build_geometry(P, G[i], src_xyz[i], nsrc[i], rec_xyz[i], nrec[i]));
        WP_TRY(dev_in(P, wavelet[i], (size_t)nsrc[i] * nt, wb[i], &wav[i]));
        WP_TRY(dev_in(P, d_obs[i], (size_t)nrec[i] * nt, ob[i], &obs[i]));
        WP_TRY(wp_malloc(P, &stage[i].p, sizeof(float) * (size_t)nt * nrec[i], "trace staging"));
        WP_TRY(wp_malloc(P, &tr[i].p, sizeof(float) * (size_t)nt * nrec[i], "traces"));
        WP_TRY(wp_malloc(P, &gb[i].p, sizeof(float) * N * 3, "gradient"));
        WP_TRY(wp_malloc(P, &gp[i].p, sizeof(float) * np * 3, "gradient (physical)"));
        WP_CK(P, cudaMemsetAsync(gb[i].p, 0, sizeof(float) * N * 3, st));
        WP_TRY(alloc_saves(P));
        WP_TRY(zero_fields(P, P->st, 9));
        WP_TRY(zero_fields(P, P->ast, 9));
        WP_TRY(zero_fields(P, P->tmp + 9, 6));     // edge and face product sums
        return PROP_OK;
    };
    for (int i = 0; i < n; i++)
        if (setup(i) != PROP_OK) {
            cudaStreamSynchronize(st);
            return 1;
        }
    const int K = ckpt_K(P0), J = ckpt_J(P0), span = ckpt_span(P0);
    if (span != nt - 1) return 1;
    for (int i = 1; i < n; i++)
        if (ckpt_K(shots[i]) != K || ckpt_J(shots[i]) != J || ckpt_span(shots[i]) != span) return 1;
    const int sf = (int)snap_fields(P0);
    DevBuf tbuf;
    WP_TRY(wp_malloc(P0, &tbuf.p, sizeof(int), "time index"));
    int *tdev = (int *)tbuf.p;
    auto g3 = [&](int i, int c) { return (float *)gb[i].p + (size_t)c * shots[i]->g.N; };
    auto xs = [&](int i, int slot, const float **out) {
        prop_s *P = shots[i];
        for (int f = 0; f < 9; f++) out[f] = f < sf ? seg_slot(P, slot) + (size_t)f * P->g.N : nullptr;
    };
    // fixed tables: slot 0 the forward step; slot 1 + p the transposed step
    // with imaging at segment position p (forward levels p and p + 1)
    std::unique_ptr<TtiBatch, void (*)(TtiBatch *)> tb(tti_batch_new(), tti_batch_free);
    std::vector<ElBatchReq> req(n);
    std::string err;
    for (int i = 0; i < n; i++) {
        req[i] = ElBatchReq{shots[i], {}, 0, 1.f, {}, {}, {}};
        for (int k = 0; k < 9; k++) req[i].S[k] = shots[i]->st[k];
    }
    if (int rc = el_batch_fix(tb.get(), req.data(), n, 0, st, &err)) return rc == 1 ? 1 : wp_fail(P0, rc, err);
    for (int pos = 0; pos < K; pos++) {
        for (int i = 0; i < n; i++) {
            req[i] = ElBatchReq{shots[i], {}, 1, 1.f, {}, {}, {g3(i, 0), g3(i, 1), g3(i, 2)}};
            for (int k = 0; k < 9; k++) req[i].S[k] = shots[i]->ast[k];
            xs(i, pos, req[i].xk);
            xs(i, pos + 1, req[i].xk1);
        }
        if (int rc = el_batch_fix(tb.get(), req.data(), n, 1 + pos, st, &err))
            return rc == 1 ? 1 : wp_fail(P0, rc, err);
    }
    auto launch = [&](int slot) -> int {
        if (el_batch_launch_fixed(tb.get(), slot, st) != PROP_OK)
            return wp_fail(P0, PROP_ECUDA, "batched elastic step launch failed");
        for (int i = 0; i < n; i++) shots[i]->kern_launches += 1;
        batch_stats[0]++;
        return PROP_OK;
    };
    constexpr int W = 8;
    struct Workers {
        cudaStream_t s[W] = {};
        cudaEvent_t fork = nullptr, join[W] = {};
        ~Workers()
        {
            for (auto x : s)
                if (x) cudaStreamDestroy(x);
            if (fork) cudaEventDestroy(fork);
            for (auto e : join)
                if (e) cudaEventDestroy(e);
        }
    } wk;
    const int nwk = std::min(W, n);
    WP_CK(P0, cudaEventCreateWithFlags(&wk.fork, cudaEventDisableTiming));
    for (int w = 0; w < nwk; w++) {
        WP_CK(P0, cudaStreamCreateWithFlags(&wk.s[w], cudaStreamNonBlocking));
        WP_CK(P0, cudaEventCreateWithFlags(&wk.join[w], cudaEventDisableTiming));
    }
    auto per_shot = [&](const std::function<int(int)> &fn) -> int {
        WP_CK(P0, cudaEventRecord(wk.fork, st));
        for (int w = 0; w < nwk; w++) WP_CK(P0, cudaStreamWaitEvent(wk.s[w], wk.fork, 0));
        int rc = PROP_OK;
        for (int i = 0; i < n && !rc; i++) {
            shots[i]->stream = wk.s[i % nwk];
            rc = fn(i);
            shots[i]->stream = st;
        }
        for (int w = 0; w < nwk; w++) {
            WP_CK(P0, cudaEventRecord(wk.join[w], wk.s[w]));
            WP_CK(P0, cudaStreamWaitEvent(st, wk.join[w], 0));
        }
        return rc;
    };
    // forward step: record d^t (trace of the stress), step, inject q^t into
    // the normal stresses (and, recomputing, keep the velocities in segment
    // buffer pos + 1), t += 1
    auto fwd = [&](bool record, int pos) -> int {
        if (record)
            WP_TRY(per_shot([&](int i) -> int {
                float *const *q = shots[i]->st;
                sp_record(shots[i], &G[i].R, q[3], q[4], q[5], 1.f, (float *)stage[i].p, tdev);
                return PROP_OK;
            }));
        WP_TRY(launch(0));
        WP_TRY(per_shot([&](int i) -> int {
            prop_s *P = shots[i];
            float *const *q = P->st;
            sp_inject(P, &G[i].S, wav[i], nt, 0, P->g.dt, 0, q[3], q[4], q[5], nullptr, nullptr, tdev);
            if (pos >= 0)
                for (int f = 0; f < sf; f++)
                    WP_CK(P, cudaMemcpyAsync(seg_slot(P, pos + 1) + (size_t)f * P->g.N, q[f], P->g.N * 4,
                                             cudaMemcpyDeviceToDevice, P->stream));
            return PROP_OK;
        }));
        k_tick(P0, tdev, 1);
        return PROP_OK;
    };
    // transposed step k = t - 1 with imaging at position pos: t -= 1, the
    // pointwise kernel before, the three passes, the face products, the
    // residual r^k
    auto adj = [&](int pos) -> int {
        k_tick(P0, tdev, -1);
        WP_TRY(per_shot([&](int i) -> int {
            el_adj_pre_launch(shots[i], shots[i]->ast, shots[i]->stream);
            return PROP_OK;
        }));
        WP_TRY(launch(1 + pos));
        WP_TRY(per_shot([&](int i) -> int {
            prop_s *P = shots[i];
            const float *x0[9], *x1[9];
            xs(i, pos, x0);
            xs(i, pos + 1, x1);
            el_face2_launch(P, P->ast, x0, x1, P->stream);
            float *const *a = P->ast;
            sp_inject(P, &G[i].R, (const float *)tr[i].p, nt, 0, 1.f, 0, a[3], a[4], a[5], nullptr, nullptr, tdev);
            return PROP_OK;
        }));
        return PROP_OK;
    };
    const char *ge = getenv("WAVEPROP_GRAPHS");
    const bool graphs = !(ge && !strcmp(ge, "0"));
    struct Graphs {
        cudaStream_t st;
        cudaGraphExec_t g[2] = {};
        ~Graphs()
        {
            cudaStreamSynchronize(st);
            for (auto e : g)
                if (e) cudaGraphExecDestroy(e);
        }
    } gx{st};
    std::vector<long long> held[2];     // launches each graph holds, per shot
    auto run = [&](int id, const std::function<int()> &body) -> int {
        if (!graphs) return body();
        if (!gx.g[id]) {
            std::vector<long long> before(n);
            for (int i = 0; i < n; i++) before[i] = shots[i]->kern_launches;
            cudaGraph_t gr = nullptr;
            WP_CK(P0, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int rb = body();
            const cudaError_t ec = cudaStreamEndCapture(st, &gr);
            if (rb || ec != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                cudaGetLastError();
                return rb ? rb : wp_cuda(P0, ec, "capture of the lockstep segment");
            }
            const cudaError_t ei = cudaGraphInstantiate(&gx.g[id], gr, 0);
            cudaGraphDestroy(gr);
            WP_CK(P0, ei);
            held[id].resize(n);
            for (int i = 0; i < n; i++) held[id][i] = shots[i]->kern_launches - before[i];
        } else {
            for (int i = 0; i < n; i++) shots[i]->kern_launches += held[id][i];
        }
        WP_CK(P0, cudaGraphLaunch(gx.g[id], st));
        return PROP_OK;
    };
    // ---- forward sweep with checkpoints ----
    k_set_int(P0, tdev, 0);
    for (int j = 0; j < J; j++) {
        const int n0 = j * K, n1 = j + 1 < J ? n0 + K : nt;
        WP_TRY(per_shot([&](int i) -> int { return save_checkpoint(shots[i], j, shots[i]->st); }));
        auto body = [&]() -> int {
            for (int t = n0; t < n1; t++) WP_TRY(fwd(true, -1));
            return PROP_OK;
        };
        if (n1 - n0 == K) WP_TRY(run(0, body));
        else WP_TRY(body());
    }
    // ---- residuals and misfits ----
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        const long long m = (long long)nrec[i] * nt;
        sp_transpose(P, (const float *)stage[i].p, (float *)tr[i].p, nrec[i], nt);
        k_axpy_sq(P, (const float *)tr[i].p, obs[i], (float *)tr[i].p, m);
        double ss = 0.0;
        WP_TRY(k_sumsq(P, (const float *)tr[i].p, m, &ss));
        mis[i] = 0.5 * ss;
    }
    // ---- adjoint sweep: k = nt - 1 (a transposed step of the zero state and
    // the last residual sample), then the segments, last first ----
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        float *const *a = P->ast;
        WP_TRY(el_launch_step(P, P->ast, true));
        sp_inject(P, &G[i].R, (const float *)tr[i].p, nt, nt - 1, 1.f, 0, a[3], a[4], a[5], nullptr, nullptr);
    }
    for (int j = J - 1; j >= 0; j--) {
        const int n0 = j * K, E = std::min(n0 + K, nt - 1), len = E - n0;
        WP_TRY(per_shot([&](int i) -> int {
            prop_s *P = shots[i];
            WP_TRY(load_checkpoint(P, j, P->st));
            for (int f = 0; f < sf; f++)
                WP_CK(P, cudaMemcpyAsync(seg_slot(P, 0) + (size_t)f * P->g.N, P->st[f], P->g.N * 4,
                                         cudaMemcpyDeviceToDevice, P->stream));
            return PROP_OK;
        }));
        k_set_int(P0, tdev, n0);
        auto body = [&]() -> int {
            for (int pos = 0; pos < len; pos++) WP_TRY(fwd(false, pos));
            for (int k = E - 1; k >= n0; k--) WP_TRY(adj(k - n0));
            return PROP_OK;
        };
        if (len == K) WP_TRY(run(1, body));
        else WP_TRY(body());
    }
    // ---- gradients on the physical grid ----
    for (int i = 0; i < n; i++) {
        prop_s *P = shots[i];
        const size_t np = (size_t)P->g.px * P->g.py * P->g.pz;
        float *gg[3] = {g3(i, 0), g3(i, 1), g3(i, 2)};
        WP_TRY(el_grad_gather(P, gg));
        for (int c = 0; c < 3; c++) k_fold(P, gg[c], (float *)gp[i].p + c * np, P->tmp[0], P->tmp[1]);
        WP_TRY(copy_out(P, grad[i], (const float *)gp[i].p, np * 3));
    }
    int first = PROP_OK;
    for (int i = 0; i < n; i++) {
        const int rc = finish(shots[i]);
        if (rc && !first) {
            first = rc;
            tl_err = "shot " + std::to_string(i) + ": " + prop_last_error(shots[i]);
        }
    }
    for (int i = 0; i < n; i++) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(e, st);
            cudaStreamWaitEvent(own[i], e, 0);
            cudaEventDestroy(e);
        }
    }
    return first;
}

extern "C" int prop_gradient_batch(prop_t *const *shots, int nshots, const float *const *wavelet,
                                   const float *const *src_xyz, const int *nsrc,
                                   const float *const *rec_xyz, const int *nrec,
                                   const float *const *d_obs, float *const *grad, double *misfit,
                                   size_t budget_bytes)
{
    if (nshots < 0) return wp_fail(nullptr, PROP_EINVAL, "nshots < 0");
    if (nshots == 0) return PROP_OK;
    if (!shots || !wavelet || !src_xyz || !nsrc || !rec_xyz || !nrec || !d_obs || !grad)
        return wp_fail(nullptr, PROP_EINVAL, "NULL array argument");
    for (int i = 0; i < nshots; i++) {
        if (!shots[i]) return wp_fail(nullptr, PROP_EINVAL, "shot handle " + std::to_string(i) + " is NULL");
        for (int j = 0; j < i; j++)
            if (shots[j] == shots[i])
                return wp_fail(nullptr, PROP_EINVAL, "shot handle " + std::to_string(i) + " repeats an earlier one");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return wp_fail(nullptr, PROP_ECUDA, "cudaGetDevice failed");
    if (budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return wp_fail(nullptr, PROP_ECUDA, "cudaMemGetInfo failed");
        budget_bytes = fr / 10 * 9;
    }
    std::vector<size_t> need(nshots);
    for (int i = 0; i < nshots; i++) need[i] = gradient_bytes(shots[i], nrec[i]);
    std::vector<int> wave(nshots);
    const int nw = prop_plan_waves(need.data(), nshots, budget_bytes, wave.data());
    std::vector<int> rc(nshots, PROP_OK);
    std::vector<double> mis(nshots, 0.0);
    batch_stats[0] = batch_stats[1] = 0;
    // shared launches for the TTI steps of a wave (WAVEPROP_BATCH_LAUNCH=0:
    // every shot launches its own)
    const char *bl = getenv("WAVEPROP_BATCH_LAUNCH");
    const bool share = !(bl && !strcmp(bl, "0"));
    const char *vb = getenv("WAVEPROP_BATCH_VERBOSE");
    const bool verbose = vb && !strcmp(vb, "1");
    for (int w = 0; w < nw; w++) {
        const auto tw = std::chrono::steady_clock::now();
        struct WaveTime {
            bool on;
            int w;
            std::chrono::steady_clock::time_point t0;
            ~WaveTime()
            {
                if (on)
                    fprintf(stderr, "wave %d: %9.3f ms\n", w,
                            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
            }
        } wt{verbose, w, tw};
        // a wave of TTI shots with one sweep: lockstep, one host thread
        std::vector<int> ids;
        for (int i = 0; i < nshots; i++)
            if (wave[i] == w) ids.push_back(i);
        std::vector<prop_t *> ws;
        for (int i : ids) ws.push_back(shots[i]);
        if (share && lockstep_ok(ws.data(), (int)ws.size())) {
            const int m = (int)ids.size();
            std::vector<const float *> wv(m), sx(m), rx(m), dob(m);
            std::vector<float *> gr(m);
            std::vector<int> ns(m), nr(m);
            std::vector<double> ms(m, 0.0);
            for (int k = 0; k < m; k++) {
                const int i = ids[k];
                wv[k] = wavelet[i]; sx[k] = src_xyz[i]; rx[k] = rec_xyz[i]; dob[k] = d_obs[i];
                gr[k] = grad[i]; ns[k] = nsrc[i]; nr[k] = nrec[i];
            }
            const int lr = (el_batchable(ws[0]) ? el_gradient_lockstep : gradient_lockstep)(
                ws.data(), m, wv.data(), sx.data(), ns.data(), rx.data(), nr.data(), dob.data(), gr.data(), ms.data());
            if (lr != 1) {
                for (int k = 0; k < m; k++) {
                    const int i = ids[k];
                    rc[i] = lr;
                    mis[i] = ms[k];
                    if (!lr) rc[i] = prop_trim(shots[i]);     // the next waves get the work arrays
                }
                continue;
            }
        }
        std::unique_ptr<StepRendezvous> rdv;
        int nb = 0;
        for (int i = 0; i < nshots; i++)
            if (wave[i] == w && (tti_batchable(shots[i]) || el_batchable(shots[i])) && !shots[i]->broken) nb++;
        if (share && nb >= 2) {
            rdv.reset(new StepRendezvous());
            if (rdv->init(nshots) != PROP_OK) rdv.reset();
            else rdv->active = nb;
        }
        for (int i = 0; i < nshots; i++)
            if (rdv && wave[i] == w && (tti_batchable(shots[i]) || el_batchable(shots[i])) && !shots[i]->broken) {
                shots[i]->rdv = rdv.get();
                shots[i]->rdv_idx = i;
            }
        std::vector<std::thread> th;
        for (int i = 0; i < nshots; i++) {
            if (wave[i] != w) continue;
            th.emplace_back([&, i] {
                prop_s *P = shots[i];
                struct Leave {       // leave the rendezvous on every way out
                    prop_s *P;
                    ~Leave()
                    {
                        if (P->rdv) {
                            P->rdv->leave();
                            P->rdv = nullptr;
                            P->rdv_idx = -1;
                        }
                    }
                } leave_rdv{P};
                if (cudaSetDevice(dev) != cudaSuccess) {
                    rc[i] = wp_fail(P, PROP_ECUDA, "cudaSetDevice failed");
                    return;
                }
                // private stream, ordered after the caller's stream and
                // before anything the caller enqueues later
                cudaStream_t own = P->stream, s = nullptr;
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
                    if (s) cudaStreamDestroy(s);
                    if (e0) cudaEventDestroy(e0);
                    rc[i] = wp_fail(P, PROP_ECUDA, "stream/event creation failed");
                    return;
                }
                cudaEventRecord(e0, own);
                cudaStreamWaitEvent(s, e0, 0);
                P->stream = s;
                P->no_tail = true;                    // concurrent shots share the free memory
                rc[i] = prop_gradient(P, wavelet[i], src_xyz[i], nsrc[i], rec_xyz[i], nrec[i], d_obs[i],
                                      grad[i], &mis[i]);
                P->no_tail = false;
                if (P->rdv) {                         // no more steps from this shot
                    P->rdv->leave();
                    P->rdv = nullptr;
                    P->rdv_idx = -1;
                }
                cudaStreamSynchronize(s);
                if (!rc[i]) rc[i] = prop_trim(P);     // the next waves get this shot's work arrays
                cudaEventRecord(e1, s);
                cudaStreamWaitEvent(own, e1, 0);
                P->stream = own;
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            });
        }
        for (auto &t : th) t.join();
        if (rdv) {
            batch_stats[0] += rdv->batched;
            batch_stats[1] += rdv->alone;
        }
    }
    int first = PROP_OK;
    for (int i = 0; i < nshots; i++) {
        if (misfit) misfit[i] = mis[i];
        if (rc[i] && !first) {
            first = rc[i];
            tl_err = "shot " + std::to_string(i) + ": " + prop_last_error(shots[i]);
        }
    }
    return first;
}
