// Internal declarations of the waveprop CUDA library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/waveprop.h"
#include "../../include/waveprop_diag.h"

#define WP_MAXM 8   // space order up to 16

// Computational grid as seen by the kernels.  Index (x,y,z) -> (x*NY + y)*NZ + z.
struct GridDev {
    int NX, NY, NZ;          // computational grid
    int nbl, px, py, pz;     // absorbing width, physical grid
    int nby;                 // absorbing width on the y faces (0 in 2D)
    long long N;             // NX*NY*NZ
    float h, ih, dt;         // spacing, 1/h, time step
    float sig0;              // TTI damping: sigma(d) = sig0 * (d/L)^2 per axis [1/s]
    float cer;               // elastic Cerjan coefficient per cell (0.015)
    // per-axis absorbing-layer tables (device):
    //   TTI:     sigma_x[NX], sigma_y[NY], sigma_z[NZ]  (sigma = sum of the three)
    //   elastic: taper_x[2 NX], taper_y[2 NY], taper_z[2 NZ]; entry 2i is the
    //            node i, 2i+1 the half point i+1/2 (taper = product of three)
    const float *tab;
};

// Finite-difference weights (FP32, from FP64 host solves).
struct FDW {
    float c[WP_MAXM];        // centred   c_1..c_M
    float b[WP_MAXM];        // staggered b_1..b_M
    float d2[WP_MAXM + 1];   // centred second derivative d2_0..d2_M (acoustic)
};

// Sparse-point tables (device).  Record: nrec x 8 (index, weight) pairs.
// Inject: unique grid cells with CSR lists of (trace, weight).
struct SparseDev {
    void *blk = nullptr;     // one device block holding the six tables below
    int n = 0;               // points
    long long *rec_idx = nullptr;
    float *rec_w = nullptr;  // [n*8]
    int ncell = 0;
    long long *cell = nullptr;
    int *cell_ptr = nullptr; // [ncell+1]
    int *ent_trace = nullptr;
    float *ent_w = nullptr;
};

struct prop_s {
    prop_desc d{};
    GridDev g{};
    FDW w{};
    int M = 0;
    cudaStream_t stream = nullptr;
    bool broken = false;
    std::string err;
    float vmax = 0.f;        // max model velocity used for the CFL rule
    // model (computational grid)
    float *m = nullptr, *eps = nullptr, *del = nullptr, *th = nullptr, *ph = nullptr;   // TTI
    float *acw = nullptr;    // acoustic: dt^2 / m
    float *nrm[2] = {};      // TTI symmetry axis n_x, n_y (sign chosen so that n_z >= 0)
    float *bu = nullptr, *lam = nullptr, *mu = nullptr;                                 // elastic
    // state: TTI 4 fields (p_cur, r_cur, p_prev, r_prev); elastic 9 fields
    float *st[9] = {};
    // scratch: TTI 6 intermediates (ex ey ez fx fy fz) + 2 (zeta p, r);
    // elastic adjoint: 6 (stress-like) + 3 (weighted velocity) + 6 gradient
    // products (edges xy xz yz, faces x y z)
    float *tmp[20] = {};
    int *flag = nullptr;     // device: bit0 NaN/Inf seen, bit1 a bounded wait expired
    double *sumsq = nullptr; // device: partial sums of k_sumsq (kept between calls)
    float *tab = nullptr;    // per-axis absorbing-layer tables (GridDev::tab)
    int xchunk = 8;          // planes per CTA of the x-streaming stencil kernels
    int tile_y = 16;         // rows (y) per tile of the TMA-fed passes: 8, 16 or 32
    // saved forward run for prop_backward
    bool saved = false;
    bool aniso = false;      // TTI gradient also w.r.t. eps, delta (prop_gradient_aniso)
    int saved_nsrc = 0, saved_nrec = 0;
    std::vector<float> saved_src, saved_rec, saved_wav;   // host copies of geometry/wavelet
    // snapshot storage
    float *snap = nullptr;   size_t snap_bytes = 0;       // full FP32 store or FP32 checkpoints
    uint16_t *snap16 = nullptr; size_t snap16_bytes = 0;  // BF16/FP16 checkpoints
    float *snap_scale = nullptr;                          // per checkpoint field scales
    float *seg = nullptr;   size_t seg_bytes = 0;         // recompute segment buffer
    // FP32 checkpoints: the last tail_T levels kept in full (sized from the
    // free device memory at the forward run; none inside batches)
    float *tail = nullptr;  size_t tail_bytes = 0;
    int tail_T = 0;
    bool no_tail = false;
    // timing of stencil kernels in the last call
    double kern_ms = 0.0;
    long long kern_launches = 0;
    bool prof = false;                                    // per-launch event timing on
    std::vector<cudaEvent_t> prof_ev;                     // pool (pairs)
    std::vector<int> prof_id;                             // id of each recorded pair
    int prof_used = 0;
    double prof_ms[8] = {};
    long long prof_n[8] = {};
    // adjoint state (separate from the forward state during gradients)
    float *ast[9] = {};
    // TMA descriptors of the stencil passes, keyed by (array, box width, box
    // height) (stencil_tma.cu)
    std::map<std::tuple<const void *, int, int>, CUtensorMap> tmaps;
    // prop_step: two steps captured as a CUDA graph, replayed; valid for the
    // state buffers, direction and tile size it was captured with
    cudaGraphExec_t step_graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    int graph_adj = -1, graph_xc = 0, graph_ty = 0;
    long long graph_launches = 0;   // kernels in one replay
    float *graph_st[9] = {};
    // batched shots: the TTI steps of this handle meet those of the other
    // shots of its wave and share one launch per pass (prop_gradient_batch)
    struct StepRendezvous *rdv = nullptr;
    int rdv_idx = -1;
};

// ---------------------------------------------------------------------------
// kernels (launchers), one translation unit per family
// ---------------------------------------------------------------------------
// TTI step on state S = (p_cur, r_cur, p_prev, r_prev): the new level is
// written over (p_prev, r_prev).  adjoint: transposed step on the adjoint
// state (lam^{k+1}, lam^{k+2}); with grad != NULL also the imaging term using
// the forward wavefield (img_p, img_r) at the new level.
int tti_launch_step(prop_s *P, float *const *S, bool adjoint, const float *img_p,
                    const float *img_r, float *grad);
int tti_launch_fast(prop_s *P, float *const *S, bool adjoint, const float *img_p,
                    const float *img_r, float *grad);
// the same step with the staggered-pair operators (desc.tti_operator = 1)
int tti_sp_launch(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                  float *grad);
int tti_sp_launch_tma(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r,
                      float *grad);
// eps, delta (and tilt/azimuth) imaging of one transposed staggered-pair step
// (zeta = C lam in tmp[6], tmp[7]; uses tmp[0..5], tmp[8..19])
int tti_sp_image_aniso_tma(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr,
                           float *ge, float *gd, float *const *gax);
// centred first derivatives D p (dp[0..2]), D r (dr[0..2]) and the products
// of the staggered derivatives at the half points, h_i = (D+_i p)(D+_i r),
// in one TMA rotation pass
int tti_raw_half_tma(prop_s *P, const float *p, const float *r, float *const *dp, float *const *dr,
                     float *const *h);
// elastic step in place on S (9 fields); adjoint: transposed step (tbar form)
int el_launch_step(prop_s *P, float *const *S, bool adjoint);
// pipelined elastic step with time step dt_sign * dt (any NZ): forward (+1)
// or the transposed step in (b_avg vbar, g C tbar) variables (-1)
int el_launch_fast(prop_s *P, float *const *S, float dt_sign);
// one 2D elastic step of S = (vx, vz, txx, tzz, txz); dt_sign = -1: the
// transposed step in the adjoint-modelling variables
int el2_launch(prop_s *P, float *const *S, float dt_sign);
// TMA-fed passes (stencil_tma.cu): usable when NZ % 4 == 0
bool tma_usable(const prop_s *P);
// acoustic step (S[0] = u^n, S[1] = u^{n-1} <- u^{n+1}); grad != NULL:
// transposed step with imaging grad -= dt^2 uf (L lam) / m
int acu_launch_step(prop_s *P, float *const *S, const float *uf, float *grad);
int acu_launch_tma(prop_s *P, float *const *S, const float *uf, float *grad);
// bounded-wait self-test: a wait that nothing completes, limit in seconds
int wait_probe_launch(prop_s *P, double seconds);
int el_launch_tma(prop_s *P, float *const *S, float dt_sign);
// true if the handle's TMA passes can run at a tile height of ty rows (8, 16,
// 32: elastic and centred TTI; 16 only for the other kinds)
bool tile_height_fits(const prop_s *P, int ty);
// TTI imaging of the coupling matrix (TMA passes): with the forward field
// (up, ur) at level n and the adjoint field (lp, lr) at level n+1,
// ge += 2 dt^2 lam_p H0 p^n, gd += dt^2 (lam_p Hz r^n + lam_r H0 p^n) / sqrt(1+2 delta)
// gax != NULL (3 fields): also gax += dt^2 V, V the dJ/dn term of the step
// (tilt/azimuth imaging; zeta = C lam must be in tmp[6], tmp[7]; uses tmp[0..13])
int tti_image_aniso_tma(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr,
                        float *ge, float *gd, float *const *gax);
// the same imaging on the pipelined passes (any NZ, centred operators);
// forms zeta = C lam itself (tmp[6], tmp[7]); uses tmp[0..13]
int tti_image_aniso_fast(prop_s *P, const float *up, const float *ur, const float *lp, const float *lr,
                         float *ge, float *gd, float *const *gax);
// pointwise tilt/azimuth term: acc += dt^2 V from the raw derivatives dz of
// zeta and du of the forward field (6 fields each)
void tti_axis_image_launch(prop_s *P, const float *const *dz, const float *const *du, float *const *acc);
// dJ/dn accumulators a[0..2] -> dJ/dtheta in a[0], dJ/dphi in a[1] (pointwise)
void tti_axis_to_angles(prop_s *P, float *const *a);
// TMA passes of a transposed elastic step with imaging: on entry S[3..8] hold
// t = g tbar and sig[0..5] = C t; updates vbar (S[0..2]), writes b_avg vbar to
// w[0..2], accumulates g_lambda, g_mu (gr[0], gr[1]) and the edge products
// ep[0..2] with the strain of v1 (forward velocities at k+1), then
// tbar = t - dt S(w) into S[3..8]
int el_adj_grad_tma(prop_s *P, float *const *S, float *const *sig, float *const *w, const float *const *v1,
                    float *const *gr, float *const *ep);
int tti_launch_tma(prop_s *P, float *const *S, bool adjoint, const float *img_p,
                   const float *img_r, float *grad);
// transposed elastic step in the variables (b_avg vbar, g C tbar): the
// forward step with dt -> -dt
int el_step_adjoint_u(prop_s *P, float *const *S);

// batched TTI steps (stencil_tma.cu): one rotation and one update launch for
// the steps of several shots (TMA path, centred operators, same space order
// and step kind).  A request is one shot's step as tti_launch_step takes it.
struct TtiBatchReq {
    prop_s *P;
    float *S[4];
    bool adjoint;
    const float *up, *ur;
    float *grad;
};
struct TtiBatch;             // device tables and host staging of a batch
TtiBatch *tti_batch_new();
void tti_batch_free(TtiBatch *b);
// 0: launched on `stream`; 1: the requests cannot share a launch (the caller
// launches them one by one); < 0: error (message in *err)
int tti_batch_step(TtiBatch *b, const TtiBatchReq *req, int n, cudaStream_t stream, std::string *err);
// step configuration `slot` (any index >= 0; forward, transposed, or
// transposed with imaging, as the requests say) of every request into a
// fixed device table (1: not batchable); then launches of that table, which
// may be captured into a CUDA graph (no host staging)
int tti_batch_fix(TtiBatch *b, const TtiBatchReq *req, int n, int slot, cudaStream_t stream, std::string *err);
int tti_batch_launch_fixed(TtiBatch *b, int slot, cudaStream_t stream);
// true if the handle's TTI steps can join a batched launch
bool tti_batchable(const prop_s *P);
// batched elastic steps: mode 0 a step with time step sign * dt (forward
// modelling +1, adjoint modelling -1); mode 1 the transposed step with
// imaging of el_launch_adj_grad (S, xk, xk1, g as there)
struct ElBatchReq {
    prop_s *P;
    float *S[9];
    int mode;
    float sign;
    const float *xk[9], *xk1[9];
    float *g[3];
};
bool el_batchable(const prop_s *P);
// 0 launched; 1 not batchable together (launch one by one); < 0 error
int el_batch_step(TtiBatch *b, const ElBatchReq *req, int n, cudaStream_t stream, std::string *err);
// fixed table `slot` of an elastic step of every request (mode 0 with sign
// +1, or mode 1: the three passes of the transposed step with imaging,
// without its pointwise kernels; 1: not batchable), and launches of it that
// may be captured
int el_batch_fix(TtiBatch *b, const ElBatchReq *req, int n, int slot, cudaStream_t stream, std::string *err);
int el_batch_launch_fixed(TtiBatch *b, int slot, cudaStream_t stream);
// per-shot pointwise kernels of the batched transposed elastic step (elastic.cu)
void el_adj_pre_launch(prop_s *P, float *const *S, cudaStream_t st);
void el_face2_launch(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1, cudaStream_t st);
int rdv_el_step(prop_s *P, const ElBatchReq &r);
// a TTI step of a shot taking part in a rendezvous (runtime.cu): waits for
// the other shots of the wave and shares their launch
int rdv_tti_step(prop_s *P, float *const *S, bool adjoint, const float *img_p, const float *img_r, float *grad);

// sparse ops (sparse.cu)
// Host-side trilinear tables of n points (metres, origin at the first
// physical point): per point 8 (index, weight) pairs, zero weights dropped
// (rec_*), and the unique cells with CSR lists of (trace, weight) (cells, ptr,
// trs, ws) for injection.  trace_of_point == NULL: trace i for point i.
struct SpHost {
    std::vector<long long> ridx, cells;
    std::vector<float> rw, ws;
    std::vector<int> ptr, trs;
};
int sp_host_tables(prop_s *P, const float *xyz_host, int n, const int *trace_of_point, SpHost &T);
// device copy of the tables in one allocation (wp_malloc); sp_free releases it
int sp_build(prop_s *P, const float *xyz_host, int n, const int *trace_of_point, SparseDev *S);
void sp_free(SparseDev *S);
// record: out[t*n + i] = scale * sum_c w * (f0 + f1 + f2)[idx]   (f1, f2 may be NULL);
// out_col is the column of step t, or with tdev the base of the [nt][n]
// staging array and t read from device memory (graph replay)
void sp_record(prop_s *P, const SparseDev *S, const float *f0, const float *f1, const float *f2,
               float scale, float *out_col, const int *tdev = nullptr);
// device time index += d (one thread; steps replayed from a CUDA graph)
void k_tick(prop_s *P, int *tdev, int d);
void k_set_int(prop_s *P, int *p, int v);
// inject: f[cell] += coef(cell) * sum_j w_j traces[trace_j*nt + t] into up to 3 fields;
// mode 0: coef = scale; mode 1: coef = scale / A (TTI, A = m(1+sig dt/2));
// mode 2: coef = scale (3 lambda + 2 mu) (elastic adjoint in s = C tbar);
// mode 3: as mode 1 into f0 = lam_p, and (1 + 2 eps), sqrt(1 + 2 delta) times
// that into f1 = zeta_p, f2 = zeta_r (TTI transposed step, zeta = C lam);
// grad_u != NULL: grad[cell] -= u[cell] * scale*sum / m  (TTI imaging of the
// residual injection)
// (tdev != NULL: t read from device memory)
void sp_inject(prop_s *P, const SparseDev *S, const float *traces, int nt, int t, float scale,
               int mode, float *f0, float *f1, float *f2, const float *grad_u, float *grad,
               const int *tdev = nullptr);
// as sp_record but each field sum is divided by (3 lambda + 2 mu) at the cell
// (trace of tbar from s = C tbar)
void sp_record_trace_s(prop_s *P, const SparseDev *S, const float *f0, const float *f1,
                       const float *f2, float scale, float *out_col);
void sp_transpose(prop_s *P, const float *in_tn, float *out_nt, int n, int nt);

// misc kernels
void k_extend(prop_s *P, const float *phys, float *comp, float scale, int mode);
// fold a computational-grid array onto the physical grid (transpose of the
// edge-replication extension); s1, s2: scratch of N floats each
void k_fold(prop_s *P, const float *comp, float *phys, float *s1, float *s2);
void k_axpy_sq(prop_s *P, const float *a, const float *b, float *out, long long n);
// sum of squares of n device floats, summed in FP64 on the host; errors of
// the allocation, launch or copy are returned (the handle keeps the buffer)
int k_sumsq(prop_s *P, const float *a, long long n, double *out);
void k_tti_zeta(prop_s *P, const float *lp, const float *lr, float *zp, float *zr);
// out = s / a (pointwise, n values)
void k_ratio(prop_s *P, const float *a, float s, float *out, long long n);
// stack[off + (i, j, k)] += weight * img[i][j][k] over the handle's physical grid
void k_stack(prop_s *P, const float *img, float *stack, const int *gdims, const int *off, float weight);
// snapshot codec
void k_snap_encode(prop_s *P, const float *in, long long n, uint16_t *out, float *scale_dev,
                   int bf16, float *scratch);
void k_snap_decode(prop_s *P, const uint16_t *in, long long n, const float *scale_dev,
                   int bf16, float *out);
// elastic transposed step fused with the gradient of forward step k:
// xk = X^k, xk1 = X^{k+1} (9 fields each), g = (g_lambda, g_mu, g_b) accumulated
// gather the edge and face products summed in tmp[9..14] over a sweep onto
// the nodes: g[1] (mu) and g[2] (b)
int el_grad_gather(prop_s *P, float *const *g);
int el_launch_adj_grad(prop_s *P, float *const *S, const float *const *xk, const float *const *xk1,
                       float *const *g);

// optional per-kernel timing (CUDA events on the handle's stream); ids:
// 0 TTI forward step, 1 TTI adjoint step, 2 elastic forward step,
// 3 elastic adjoint step, 4 elastic adjoint+gradient step
void prof_begin(prop_s *P, int id);
void prof_end(prop_s *P, int id);
void k_lame(prop_s *P);
void k_normals(prop_s *P);

// FD weights from the moment conditions (FP64 solve, FP32 result) and the
// maximum of the discrete derivative symbol (CFL bound)
bool fd_weights(int M, float *c, float *bst);
double symbol_max(const float *w, int M, bool stag);
// host: per-axis absorbing-layer tables (layout of GridDev::tab)
std::vector<float> layer_tables(const GridDev &g, int kind);
// planes per CTA for the x-streaming stencil kernels
int stencil_xchunk(const GridDev &g, int sms);

// error helpers
int wp_fail(prop_s *P, int code, const std::string &msg);
// every device allocation of the library goes through wp_dev_alloc
// (WAVEPROP_FAULT=alloc: every allocation fails): PROP_ENOMEM or PROP_ECUDA
// with the message in *msg (may be NULL), *p = NULL on failure; wp_malloc
// records the failure on the handle (P may be NULL)
int wp_dev_alloc(void **p, size_t bytes, const char *what, std::string *msg);
int wp_malloc(prop_s *P, void **p, size_t bytes, const char *what);
// status of the device error word read back after a call: bit 3 (the
// bounds-checking build skipped an access) -> PROP_ECUDA; bit 1 (a bounded
// device wait expired) -> PROP_ETIMEOUT; bit 0 (NaN/Inf seen) ->
// PROP_EUNSTABLE when check_nan is set; else PROP_OK
int wp_flag_status(prop_s *P, int flag);
int wp_cuda(prop_s *P, cudaError_t e, const char *what);
#define WP_CK(P, call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return wp_cuda((P), _e, #call);  \
    } while (0)
#define WP_TRY(expr)                 \
    do {                             \
        int _r = (expr);             \
        if (_r) return _r;           \
    } while (0)
