// Host runtime of the lbm2p C ABI: parameter checks, device memory, the physical-step
// driver and the pressure sub-iteration control (Sec. 3).  Every lattice operation runs
// in the kernels of kernels.cu; this file only validates, uploads, launches and reads back.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm2p.h"
#include "lbm2p_device.cuh"
#include "lbm2p_handle.h"

using namespace lbm2p_dev;

namespace {

thread_local std::string g_create_error;
constexpr int kStatePlanes = 20;   // n_1..n_8, g_0..g_8, 1/tau_f, S, R
using lbm2p_internal::Alloc;

}  // namespace

namespace lbm2p_internal {

// ---- kernel argument blocks --------------------------------------------------------------
PressureArgs pressure_args(lbm2p *h, int src, int dst, bool work)
{
    PressureArgs a{};
    for (int i = 0; i < 8; ++i) {
        a.fin[i] = h->fbuf[src][i];
        a.fout[i] = h->fbuf[dst][i];
    }
    a.R = R_of(h, work);
    a.inv_tau = itau_of(h, work);
    a.Fp = h->Fp;
    a.Pio = h->Pio;
    a.partials = h->partials;
    a.shift = h->shift;
    for (int s = 0; s < 4; ++s)
        a.Pb[s] = h->Pb[s];
    a.g = h->geom;
    a.w = h->wells;
    return a;
}

RefreshArgs refresh_args(lbm2p *h, int pg, bool in_place)
{
    RefreshArgs a{};
    for (int i = 0; i < 9; ++i)
        a.gin[i] = h->gbuf[pg][i];
    a.Rin = R_of(h, false);
    a.Rout = R_of(h, !in_place);
    a.Pstep_in = h->p.warm_start ? Pstep_of(h, false) : nullptr;
    a.Pstep_out = h->p.warm_start ? Pstep_of(h, !in_place) : nullptr;
    a.K = h->K;
    a.Fs = h->Fs;
    a.inv_tau = itau_of(h, !in_place);
    for (int s = 0; s < 4; ++s)
        a.Sb[s] = h->Sb[s];
    a.g = h->geom;
    a.m = h->model;
    a.w = h->wells;
    return a;
}

SaturationArgs saturation_args(lbm2p *h, int pf, int pg, bool work)
{
    SaturationArgs a{};
    for (int i = 0; i < 8; ++i)
        a.fin[i] = h->fbuf[pf][i];
    a.R = R_of(h, work);
    a.Pnew = h->Pio;
    for (int i = 0; i < 9; ++i) {
        a.gin[i] = h->gbuf[pg][i];
        a.gout[i] = h->gbuf[1 - pg][i];
    }
    a.K = h->K;
    a.inv_tau = itau_of(h, work);
    a.Fs = h->Fs;
    a.S = h->S;
    for (int s = 0; s < 4; ++s) {
        a.Pb[s] = h->Pb[s];
        a.Sb[s] = h->Sb[s];
    }
    a.g = h->geom;
    a.m = h->model;
    a.w = h->wells;
    return a;
}


RebaseMidArgs rebase_mid_args(lbm2p *h, int pf, bool work)
{
    RebaseMidArgs a{};
    for (int i = 0; i < 8; ++i)
        a.n[i] = h->fbuf[pf][i];
    a.R = R_of(h, work);
    a.Fp = h->Fp;
    a.g = h->geom;
    a.w = h->wells;
    return a;
}

RebaseArgs rebase_args(lbm2p *h, int pf, bool work)
{
    RebaseArgs a{};
    for (int i = 0; i < 8; ++i)
        a.n[i] = h->fbuf[pf][i];
    a.R = R_of(h, work);
    a.Pnew = h->Pio;
    a.g = h->geom;
    return a;
}

}  // namespace lbm2p_internal

namespace {

using lbm2p_internal::pressure_args;
using lbm2p_internal::refresh_args;
using lbm2p_internal::saturation_args;
using lbm2p_internal::rebase_args;
using lbm2p_internal::rebase_mid_args;
using lbm2p_internal::fnext;
using lbm2p_internal::itau_of;
using lbm2p_internal::R_of;
using lbm2p_internal::Pstep_of;

lbm2p_status fail(lbm2p *h, lbm2p_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CUDA_TRY(h, call)                                                                    \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((h), LBM2P_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

lbm2p_status launched(lbm2p *h, const char *what)
{
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(h, LBM2P_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return LBM2P_OK;
}

#define LAUNCHED(h, what)                                                                    \
    do {                                                                                     \
        lbm2p_status st_ = launched((h), (what));                                            \
        if (st_ != LBM2P_OK)                                                                 \
            return st_;                                                                      \
    } while (0)

void *dev_alloc(lbm2p *h, size_t bytes)
{
    void *ptr = nullptr;
    if (h->p.alloc) {
        ptr = h->p.alloc(bytes, h->p.alloc_ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr)
        h->allocs.push_back({ptr, bytes});
    return ptr;
}

// destroy the instantiated solve and step graphs (they are rebuilt on first use)
void drop_graphs(lbm2p *h)
{
    for (int a = 0; a < 3; ++a)
        for (int r = 0; r < 2; ++r) {
            if (h->solve_x[a][r])
                cudaGraphExecDestroy(h->solve_x[a][r]);
            if (h->solve_g[a][r])
                cudaGraphDestroy(h->solve_g[a][r]);
            h->solve_x[a][r] = nullptr;
            h->solve_g[a][r] = nullptr;
            for (int b = 0; b < 2; ++b) {
                if (h->step_x[a][b][r])
                    cudaGraphExecDestroy(h->step_x[a][b][r]);
                if (h->step_g[a][b][r])
                    cudaGraphDestroy(h->step_g[a][b][r]);
                h->step_x[a][b][r] = nullptr;
                h->step_g[a][b][r] = nullptr;
            }
        }
}

void free_all(lbm2p *h)
{
    for (auto &a : h->allocs) {
        if (h->p.alloc && h->p.release)
            h->p.release(a.ptr, a.bytes, h->p.alloc_ctx);
        else if (!h->p.alloc)
            cudaFree(a.ptr);
    }
    drop_graphs(h);
    h->allocs.clear();
    if (h->res_host)
        cudaFreeHost(h->res_host);
    h->res_host = nullptr;
    if (h->ctl_host)
        cudaFreeHost(h->ctl_host);
    h->ctl_host = nullptr;
    if (h->hscale_host)
        cudaFreeHost(h->hscale_host);
    h->hscale_host = nullptr;
    for (cudaEvent_t *e : {&h->ev_step0, &h->ev_step1, &h->ev_sw0, &h->ev_sw1})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
}

// lambda_t at S for the model (host, FP64; used for D_ref only)
double lambda_t_host(const lbm2p_params &p, double S)
{
    if (p.mobility == LBM2P_MOB_QUADRATIC)
        return S * S / p.mu_w + (1.0 - S) * (1.0 - S) / p.mu_n;
    if (p.mobility == LBM2P_MOB_DECOUPLED)
        return 1.0 / p.mu_w;
    return 1.0 / (0.5 - 0.2 * S);
}

int trace_len(const lbm2p *h, int side) { return side < 2 ? 2 * h->ny + 1 : 2 * h->nx + 1; }

// host FP64 [ny][nx] -> device pitched FP32 plane, with a scale factor
lbm2p_status upload_plane(lbm2p *h, float *dst, const double *src, double scale)
{
    std::vector<float> tmp((size_t)h->nnodes);
    for (long long a = 0; a < h->nnodes; ++a)
        tmp[(size_t)a] = (float)(scale * src[a]);
    CUDA_TRY(h, cudaMemcpy2DAsync(dst, (size_t)h->pitch * sizeof(float), tmp.data(),
                                  (size_t)h->nx * sizeof(float), (size_t)h->nx * sizeof(float),
                                  (size_t)h->ny, cudaMemcpyHostToDevice, (cudaStream_t)h->stream));
    CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)h->stream));
    return LBM2P_OK;
}

lbm2p_status upload_trace(lbm2p *h, float *dst, const double *src, int n)
{
    std::vector<float> tmp((size_t)n, 0.0f);
    if (src)
        for (int k = 0; k < n; ++k)
            tmp[(size_t)k] = (float)src[k];
    CUDA_TRY(h, cudaMemcpyAsync(dst, tmp.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice,
                                (cudaStream_t)h->stream));
    CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)h->stream));
    return LBM2P_OK;
}

// ---- single pressure sweeps with the kernel chosen at create ---------------------------
void launch_sweep(lbm2p *h, const PressureArgs &a, bool check, bool write_p)
{
    if (h->sweep_kind == 2)
        lbm2p_launch::pressure_sweep_rows(a, check, write_p, h->rows_w, h->rows_slots, h->rows_H,
                                          h->rows_grid, h->stream);
    else
        lbm2p_launch::pressure_sweep(a, check, write_p, check ? h->grid_check : h->grid_sweep, h->stream,
                                     h->sweep_kind);
}

cudaError_t add_sweep_node(lbm2p *h, cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                           const PressureArgs &a, bool check, bool write_p)
{
    if (h->sweep_kind == 2)
        return lbm2p_launch::node_pressure_rows(n, g, dep, a, check, write_p, h->rows_w,
                                                h->rows_slots, h->rows_H, h->rows_grid);
    return lbm2p_launch::node_pressure(n, g, dep, a, check, write_p,
                                       check ? h->grid_check : h->grid_sweep, h->sweep_kind);
}

// residual partials written by one checking single sweep
int sweep_nparts(const lbm2p *h)
{
    return h->sweep_kind == 2 ? h->rows_grid : h->grid_check;
}

// ---- graph-resident sub-iteration ----------------------------------------------------------
// Appends to G: reset(ctl) -> event(sw0) -> the first check period -> WHILE{ further check
// periods } -> event(sw1).  A check period is m = check_every sweeps (single or fused
// launches), the last with residual partials, then the finalize kernel (it counts the sweeps,
// keeps r, decides whether the WHILE goes on and whether R first moves to the current P:
// IF{mid-solve rebase}).  The first period reads f buffer pin and writes the next buffer of the
// rotation, then ping-pongs between the two buffers other than pin and ends on the third; every
// later period starts and ends there (m, or m / T fused launches, is even).  So the state the
// solve starts from is only read, and the solve ends in buffer fnext(pin, 2).  `work`: R and
// 1/tau_f of the work buffers (a step's solve) or the current ones (a bare solve).
lbm2p_status add_loop(lbm2p *h, cudaGraph_t G, const cudaGraphNode_t *dep, int pin, bool work,
                      cudaGraphNode_t *last)
{
    const int m = h->p.check_every;
    const int b1 = fnext(pin, 1), b2 = fnext(pin, 2);
    auto dst_of = [&](int src) { return src == b1 ? b2 : b1; };
    cudaGraphNode_t reset, ev0, first_end, wn, ev1;
    CUDA_TRY(h, lbm2p_launch::node_loop_reset(&reset, G, dep, h->ctl));
    CUDA_TRY(h, cudaGraphAddEventRecordNode(&ev0, G, &reset, 1, h->ev_sw0));
    cudaGraphConditionalHandle hd;
    CUDA_TRY(h, cudaGraphConditionalHandleCreate(&hd, G, 1, cudaGraphCondAssignDefault));
    // one check period into graph g after node `after` (nullptr: none), its first launch
    // reading buffer `first`, the mid-solve rebase conditioned on handle hr
    auto period = [&](cudaGraph_t g, cudaGraphNode_t after, int first,
                      cudaGraphConditionalHandle hr, cudaGraphNode_t *out) -> lbm2p_status {
        cudaGraphNode_t prev = after;
        int src = first;
        int nparts = sweep_nparts(h);
        if (h->tb_T_graph > 1) {
            const int T = h->tb_T_graph;
            for (int kk = T; kk <= m; kk += T) {
                cudaGraphNode_t n;
                PressureArgs a = pressure_args(h, src, dst_of(src), work);
                if (h->tb_kind == 2)
                    CUDA_TRY(h, lbm2p_launch::node_pressure_pair_direct(&n, g, prev ? &prev : nullptr,
                                                                        a, kk == m, h->tb_W / 30,
                                                                        h->tb_H, h->tb_grid));
                else if (h->tb_kind == 1)
                    CUDA_TRY(h, lbm2p_launch::node_pressure_rows2(&n, g, prev ? &prev : nullptr, a,
                                                                  kk == m, h->tb_W / 30, h->tb_slots,
                                                                  h->tb_H, h->tb_grid));
                else
                    CUDA_TRY(h, lbm2p_launch::node_pressure_fused(&n, g, prev ? &prev : nullptr, a,
                                                                  T, h->tb_W, h->tb_H, kk == m,
                                                                  h->tb_grid));
                prev = n;
                src = dst_of(src);
            }
            nparts = h->tb_grid;
        } else {
            for (int kk = 1; kk <= m; ++kk) {
                cudaGraphNode_t n;
                PressureArgs a = pressure_args(h, src, dst_of(src), work);
                CUDA_TRY(h, add_sweep_node(h, &n, g, prev ? &prev : nullptr, a, kk == m,
                                           kk == m - 1));
                prev = n;
                src = dst_of(src);
            }
        }
        // finalize decides whether to continue, and whether R moves to the current P first
        cudaGraphNode_t fin, ifn, rb;
        CUDA_TRY(h, lbm2p_launch::node_finalize_loop(&fin, g, &prev, h->partials, nparts,
                                                     h->nnodes, h->shift, h->res, h->ctl, hd, hr));
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hr;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        CUDA_TRY(h, cudaGraphAddNode(&ifn, g, &fin, nullptr, 1, &ip));
        CUDA_TRY(h, lbm2p_launch::node_rebase_mid(&rb, ip.conditional.phGraph_out[0], nullptr,
                                                  rebase_mid_args(h, b2, work), h->grid));
        *out = ifn;
        return LBM2P_OK;
    };
    cudaGraphConditionalHandle hr0;
    CUDA_TRY(h, cudaGraphConditionalHandleCreate(&hr0, G, 0, 0));
    lbm2p_status e = period(G, ev0, pin, hr0, &first_end);
    if (e != LBM2P_OK)
        return e;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CUDA_TRY(h, cudaGraphAddNode(&wn, G, &first_end, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphConditionalHandle hr;
    CUDA_TRY(h, cudaGraphConditionalHandleCreate(&hr, body, 0, 0));
    cudaGraphNode_t body_end;
    if ((e = period(body, nullptr, b2, hr, &body_end)) != LBM2P_OK)
        return e;
    CUDA_TRY(h, cudaGraphAddEventRecordNode(&ev1, G, &wn, 1, h->ev_sw1));
    *last = ev1;
    return LBM2P_OK;
}

// a bare solve (current R and 1/tau_f) from f buffer pin; it ends in fnext(pin, 2)
lbm2p_status solve_graph(lbm2p *h, int pin, cudaGraphExec_t *out)
{
    const int r = h->cur_r;
    if (!h->solve_x[pin][r]) {
        cudaGraph_t G;
        CUDA_TRY(h, cudaGraphCreate(&G, 0));
        h->solve_g[pin][r] = G;
        cudaGraphNode_t last;
        lbm2p_status e = add_loop(h, G, nullptr, pin, false, &last);
        if (e != LBM2P_OK)
            return e;
        CUDA_TRY(h, cudaGraphInstantiate(&h->solve_x[pin][r], G, 0));
    }
    *out = h->solve_x[pin][r];
    return LBM2P_OK;
}

// one physical step: refresh (into the work buffers) -> loop -> IF{the residual is a number:
// saturation update -> rebase}; the step's inputs (f buffer pin, g buffer pg, the current R,
// 1/tau_f and P^{n-1}) are only read, so a step that fails leaves them as they were
lbm2p_status step_graph(lbm2p *h, int pin, int pg, cudaGraphExec_t *out)
{
    const int r = h->cur_r;
    if (!h->step_x[pin][pg][r]) {
        cudaGraph_t G;
        CUDA_TRY(h, cudaGraphCreate(&G, 0));
        h->step_g[pin][pg][r] = G;
        cudaGraphNode_t nr, last, nf, ifn, ns, nb;
        CUDA_TRY(h, lbm2p_launch::node_refresh(&nr, G, nullptr, refresh_args(h, pg, false), h->grid));
        lbm2p_status e = add_loop(h, G, &nr, pin, true, &last);
        if (e != LBM2P_OK)
            return e;
        cudaGraphConditionalHandle hok;
        CUDA_TRY(h, cudaGraphConditionalHandleCreate(&hok, G, 0, 0));
        CUDA_TRY(h, lbm2p_launch::node_if_finite(&nf, G, &last, h->ctl, hok));
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hok;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        CUDA_TRY(h, cudaGraphAddNode(&ifn, G, &nf, nullptr, 1, &ip));
        cudaGraph_t tail = ip.conditional.phGraph_out[0];
        const int pout = fnext(pin, 2);
        CUDA_TRY(h, lbm2p_launch::node_saturation(&ns, tail, nullptr,
                                                  saturation_args(h, pout, pg, true), h->grid));
        CUDA_TRY(h, lbm2p_launch::node_rebase(&nb, tail, &ns, rebase_args(h, pout, true), h->grid));
        CUDA_TRY(h, cudaGraphInstantiate(&h->step_x[pin][pg][r], G, 0));
    }
    *out = h->step_x[pin][pg][r];
    return LBM2P_OK;
}

// read the loop's counters after a graph launch (synchronises the stream)
lbm2p_status read_loop(lbm2p *h, int *k, double *r, float *sweep_ms)
{
    cudaStream_t st = (cudaStream_t)h->stream;
    CUDA_TRY(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    *k = h->ctl_host->k;
    *r = h->ctl_host->r;
    const int m = h->p.check_every;
    const int per_launch = h->tb_T_graph > 1 ? h->tb_T_graph : 1;
    h->sweeps += *k;
    // reset, sweep launches, finalizes, mid-solve rebases
    h->launches += 1 + *k / per_launch + *k / m +
                   (h->rebase_every > 0 && *k > 0 ? (*k - 1) / h->rebase_every : 0);
    if (sweep_ms) {
        *sweep_ms = -1.0f;
        if (h->timing)
            CUDA_TRY(h, cudaEventElapsedTime(sweep_ms, h->ev_sw0, h->ev_sw1));
    }
    return LBM2P_OK;
}

lbm2p_status loop_status(lbm2p *h, int k, double r)
{
    if (std::isnan(r))
        return fail(h, LBM2P_ENONFINITE, "pressure residual is not finite after %d sweeps", k);
    if (!(r <= h->p.tol))
        return fail(h, LBM2P_ENOTCONVERGED, "pressure residual %.3e above tol %.3e after %d sweeps",
                    r, h->p.tol, k);
    return LBM2P_OK;
}

// ---- the pressure sub-iteration (Sec. 3) ------------------------------------------------
// replay >= 0: exactly that many sweeps; replay < 0: until r <= tol at a check or the cap.
lbm2p_status pressure_solve_h(lbm2p *h, int replay, bool work, int *k_out, double *r_out,
                             float *ms_out, int *pout);

// The sub-iteration with FP16 storage (fp16.cu): narrow the FP32 state of f buffer cur_f,
// sweep on FP16 with the same stopping rule and replay semantics as pressure_solve, widen the
// result into the next f buffer of the rotation (*pout), so the state it started from is only
// read.  `work`: R and 1/tau_f of the work buffers (a step's solve) or the current ones.
lbm2p_status pressure_solve_h(lbm2p *h, int replay, bool work, int *k_out, double *r_out,
                             float *ms_out, int *pout)
{
    cudaStream_t st = (cudaStream_t)h->stream;
    const int m = h->p.check_every;
    const int cap = h->p.max_sub_iters;
    const int pin = h->cur_f, pw = fnext(pin, 1);
    auto convert_args = [&](int hb) {
        HalfConvertArgs a{};
        for (int i = 0; i < 8; ++i) {
            a.n32[i] = h->fbuf[pin][i];
            a.n32w[i] = h->fbuf[pw][i];
            a.n16[i] = h->hbuf[hb][i];
        }
        a.R = R_of(h, work);
        a.Rw = R_of(h, work);
        a.Rh = h->Rh[hb];
        a.scale = h->hscale;
        a.g = h->geom;
        return a;
    };
    lbm2p_launch::half_narrow(convert_args(0), h->grid, h->stream);
    LAUNCHED(h, "FP16 narrow");
    h->hcur = 0;
    int k = 0;
    double r = std::nan("");
    float ms_total = 0.0f;
    lbm2p_status status = LBM2P_OK;
    auto sweeps = [&](int upto, bool final_check) -> lbm2p_status {
        if (h->timing)
            CUDA_TRY(h, cudaEventRecord(h->ev_sw0, st));
        for (int kk = k + 1; kk <= upto; ++kk) {
            HalfSweepArgs a{};
            for (int i = 0; i < 8; ++i) {
                a.nin[i] = h->hbuf[h->hcur][i];
                a.nout[i] = h->hbuf[1 - h->hcur][i];
            }
            a.Rin = h->Rh[h->hcur];
            a.Rout = h->Rh[1 - h->hcur];
            a.inv_tau = itau_of(h, work);
            a.Fp = h->Fp;
            a.partials = h->partials;
            a.shift = h->shift;
            a.scale = h->hscale;
            a.scale_out = h->hscale;
            for (int s = 0; s < 4; ++s)
                a.Pb[s] = h->Pb[s];
            a.g = h->geom;
            a.w = h->wells;
            const bool check = final_check && kk == upto;
            if (h->h16_kind == 1)
                lbm2p_launch::pressure_sweep_rows_h(a, check, h->h16_w, h->h16_slots, h->h16_H,
                                                    h->h16_grid, h->stream);
            else
                lbm2p_launch::pressure_sweep_h(a, check, h->grid_h, h->stream);
            LAUNCHED(h, "FP16 pressure sweep");
            h->hcur = 1 - h->hcur;
            h->sweeps += 1;
        }
        k = upto;
        if (h->timing) {
            float ms = 0.0f;
            CUDA_TRY(h, cudaEventRecord(h->ev_sw1, st));
            CUDA_TRY(h, cudaEventSynchronize(h->ev_sw1));
            CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev_sw0, h->ev_sw1));
            ms_total += ms;
        }
        return LBM2P_OK;
    };
    auto read_residual = [&]() -> lbm2p_status {
        lbm2p_launch::residual_finalize(h->partials, h->h16_kind == 1 ? h->h16_grid : h->grid_h,
                                        h->nnodes, h->shift, h->res, h->stream);
        LAUNCHED(h, "residual finalize");
        CUDA_TRY(h, cudaMemcpyAsync(h->res_host, h->res, sizeof(ResidualOut),
                                    cudaMemcpyDeviceToHost, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        r = h->res_host->r;
        return LBM2P_OK;
    };
    // keep the largest stored magnitude, as seen by the last check sweep, within [2^9, 2^14]
    // of FP16's 2^16: otherwise multiply every stored value by a power of two (exact)
    auto rescale = [&]() -> lbm2p_status {
        CUDA_TRY(h, cudaMemcpyAsync(h->hscale_host, h->hscale, 4 * sizeof(float),
                                    cudaMemcpyDeviceToHost, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        const float s = h->hscale_host[0], M = h->hscale_host[3];
        CUDA_TRY(h, cudaMemsetAsync(h->hscale + 3, 0, sizeof(float), st));
        if (!(M > 0.0f) || !std::isfinite(M) || (M >= 512.0f && M <= 16384.0f))
            return LBM2P_OK;
        int ex = 0;
        std::frexp(M, &ex);
        const float factor = std::ldexp(1.0f, 12 - ex);
        const float sn = s * factor;
        if (!(sn > 0.0f) || !std::isfinite(sn))
            return LBM2P_OK;
        lbm2p_launch::half_rescale(convert_args(h->hcur), factor, h->grid, h->stream);
        LAUNCHED(h, "FP16 rescale");
        h->hscale_host[0] = sn;
        h->hscale_host[1] = 1.0f / sn;
        CUDA_TRY(h, cudaMemcpyAsync(h->hscale, h->hscale_host, 2 * sizeof(float),
                                    cudaMemcpyHostToDevice, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        return LBM2P_OK;
    };
    lbm2p_status e;
    if (replay >= 0) {
        // long replays are cut into chunks of 256 sweeps ending in a check sweep, for the
        // rescale (the residual of intermediate chunks is not read)
        while (k + 256 < replay) {
            if ((e = sweeps(k + 256, true)) != LBM2P_OK)
                return e;
            if ((e = rescale()) != LBM2P_OK)
                return e;
        }
        if ((e = sweeps(replay, replay >= 2)) != LBM2P_OK)
            return e;
        if (replay >= 2) {
            if ((e = read_residual()) != LBM2P_OK)
                return e;
            if (std::isnan(r))
                status = LBM2P_ENONFINITE;
        }
    } else {
        for (;;) {
            int next = (k / m + 1) * m;
            next = next > cap ? cap : next;
            next = next < 1 ? 1 : next;
            if ((e = sweeps(next, next >= 2)) != LBM2P_OK)
                return e;
            if (k >= 2) {
                if ((e = read_residual()) != LBM2P_OK)
                    return e;
                if (std::isnan(r)) {
                    status = LBM2P_ENONFINITE;
                    break;
                }
                if (r <= h->p.tol)
                    break;
            }
            if (k >= cap) {
                status = LBM2P_ENOTCONVERGED;
                break;
            }
            if (k >= 2 && (e = rescale()) != LBM2P_OK)
                return e;
        }
    }
    lbm2p_launch::half_widen(convert_args(h->hcur), h->grid, h->stream);
    LAUNCHED(h, "FP16 widen");
    if (pout)
        *pout = pw;
    if (k_out)
        *k_out = k;
    if (r_out)
        *r_out = r;
    if (ms_out)
        *ms_out = h->timing ? ms_total : -1.0f;
    if (status == LBM2P_ENONFINITE)
        return fail(h, status, "pressure residual is not finite after %d sweeps", k);
    if (status == LBM2P_ENOTCONVERGED)
        return fail(h, status, "pressure residual %.3e above tol %.3e after %d sweeps", r,
                    h->p.tol, k);
    return LBM2P_OK;
}

// The pressure sub-iteration from f buffer cur_f.  The first sweep writes the next buffer of
// the rotation, later sweeps ping-pong between the two buffers other than cur_f, so the state
// the solve started from is only read; *pout receives the buffer holding the result (cur_f
// when no sweep ran).  `work`: R and 1/tau_f of the work buffers (a step's solve, after its S
// refresh) or the current ones (the t = 0 solve, lbm2p_pressure_sweeps).
lbm2p_status pressure_solve(lbm2p *h, int replay, bool work, int *k_out, double *r_out,
                            float *ms_out, int *pout)
{
    if (h->fp16)
        return pressure_solve_h(h, replay, work, k_out, r_out, ms_out, pout);
    cudaStream_t st = (cudaStream_t)h->stream;
    const int pin = h->cur_f, b1 = fnext(pin, 1), b2 = fnext(pin, 2);
    auto dst_of = [&](int src) { return src == b1 ? b2 : b1; };
    int src = pin;
    const int m = h->p.check_every;
    const int cap = h->p.max_sub_iters;
    double r = std::nan("");
    float ms_total = 0.0f;
    lbm2p_status status = LBM2P_OK;
    int k = 0;
    auto is_check = [&](int kk) {
        if (replay >= 0)
            return kk == replay;
        return (kk % m == 0) || kk >= cap;
    };
    // run sweeps k+1 .. upto; the last one evaluates the residual when asked
    int last_nparts = sweep_nparts(h);
    // run sweeps k+1 .. upto; the last one evaluates the residual when it is a check point.
    // With fused sweeps the batch is a few single sweeps followed by fused launches, the
    // last of which computes the residual from its final two stages.
    auto run_batch = [&](int upto) -> lbm2p_status {
        if (h->timing)
            CUDA_TRY(h, cudaEventRecord(h->ev_sw0, st));
        const int n = upto - k;
        const int T = h->tb_T;
        const int nf = (T > 1 && n >= T) ? n / T : 0;
        const int ns = n - nf * T;
        const bool final_check = is_check(upto) && upto >= 2;
        for (int i = 0; i < ns; ++i) {
            const int kk = k + 1 + i;
            const bool check = nf == 0 && is_check(kk) && kk >= 2;
            const bool write_p = nf == 0 && is_check(kk + 1) && kk + 1 >= 2;
            PressureArgs a = pressure_args(h, src, dst_of(src), work);
            launch_sweep(h, a, check, write_p);
            LAUNCHED(h, "pressure sweep");
            src = dst_of(src);
            h->sweeps += 1;
        }
        for (int q = 0; q < nf; ++q) {
            PressureArgs a = pressure_args(h, src, dst_of(src), work);
            if (h->tb_kind == 2)
                lbm2p_launch::pressure_sweeps_pair_direct(a, q == nf - 1 && final_check,
                                                          h->tb_W / 30, h->tb_H, h->tb_grid,
                                                          h->stream);
            else if (h->tb_kind == 1)
                lbm2p_launch::pressure_sweeps_rows2(a, q == nf - 1 && final_check, h->tb_W / 30,
                                                    h->tb_slots, h->tb_H, h->tb_grid, h->stream);
            else
                lbm2p_launch::pressure_sweeps_fused(a, T, h->tb_W, h->tb_H,
                                                    q == nf - 1 && final_check, h->tb_grid,
                                                    h->stream);
            LAUNCHED(h, "fused pressure sweeps");
            src = dst_of(src);
            h->sweeps += T;
        }
        last_nparts = nf > 0 ? h->tb_grid : sweep_nparts(h);
        if (h->timing)
            CUDA_TRY(h, cudaEventRecord(h->ev_sw1, st));
        k = upto;
        return LBM2P_OK;
    };
    auto read_residual = [&]() -> lbm2p_status {
        lbm2p_launch::residual_finalize(h->partials, last_nparts, h->nnodes, h->shift, h->res,
                                        h->stream);
        LAUNCHED(h, "residual finalize");
        CUDA_TRY(h, cudaMemcpyAsync(h->res_host, h->res, sizeof(ResidualOut),
                                    cudaMemcpyDeviceToHost, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
        r = h->res_host->r;
        return LBM2P_OK;
    };
    auto add_time = [&]() -> lbm2p_status {
        if (h->timing) {
            float ms = 0.0f;
            CUDA_TRY(h, cudaEventSynchronize(h->ev_sw1));
            CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev_sw0, h->ev_sw1));
            ms_total += ms;
        }
        return LBM2P_OK;
    };
    lbm2p_status e;
    if (replay < 0 && h->graph_ok && !work) {
        cudaGraphExec_t x;
        if ((e = solve_graph(h, pin, &x)) != LBM2P_OK)
            return e;
        CUDA_TRY(h, cudaGraphLaunch(x, st));
        float ms = -1.0f;
        if ((e = read_loop(h, &k, &r, &ms)) != LBM2P_OK)
            return e;
        if (k_out)
            *k_out = k;
        if (r_out)
            *r_out = r;
        if (ms_out)
            *ms_out = ms;
        if (pout)
            *pout = b2;
        return loop_status(h, k, r);
    }
    // R moves to the current P after sweep k when k is a multiple of rebase_every and the
    // solve goes on (the graph loop applies the same rule)
    const int every = h->rebase_every;
    auto rebase_mid = [&]() -> lbm2p_status {
        lbm2p_launch::rebase_mid(rebase_mid_args(h, src, work), h->grid, h->stream);
        LAUNCHED(h, "mid-solve rebase");
        return LBM2P_OK;
    };
    if (replay >= 0) {
        if (replay > 0) {
            while (k < replay) {
                int next = replay;
                if (every > 0 && (k / every + 1) * every < replay)
                    next = (k / every + 1) * every;
                if ((e = run_batch(next)) != LBM2P_OK)
                    return e;
                if ((e = add_time()) != LBM2P_OK)
                    return e;
                if (k < replay && every > 0 && k % every == 0 && (e = rebase_mid()) != LBM2P_OK)
                    return e;
            }
            if (replay >= 2) {
                if ((e = read_residual()) != LBM2P_OK)
                    return e;
                if (std::isnan(r))
                    status = LBM2P_ENONFINITE;
            }
        }
    } else {
        for (;;) {
            int next = (k / m + 1) * m;
            if (next > cap)
                next = cap;
            if (next < 1)
                next = 1;
            if ((e = run_batch(next)) != LBM2P_OK)
                return e;
            if ((e = add_time()) != LBM2P_OK)
                return e;
            if (k >= 2) {
                if ((e = read_residual()) != LBM2P_OK)
                    return e;
                if (std::isnan(r)) {
                    status = LBM2P_ENONFINITE;
                    break;
                }
                if (r <= h->p.tol)
                    break;
            }
            if (k >= cap) {
                status = LBM2P_ENOTCONVERGED;
                break;
            }
            if (every > 0 && k % every == 0 && (e = rebase_mid()) != LBM2P_OK)
                return e;
        }
    }
    if (k_out)
        *k_out = k;
    if (r_out)
        *r_out = r;
    if (ms_out)
        *ms_out = h->timing ? ms_total : -1.0f;
    if (pout)
        *pout = src;
    if (status == LBM2P_ENONFINITE)
        return fail(h, status, "pressure residual is not finite after %d sweeps", k);
    if (status == LBM2P_ENOTCONVERGED)
        return fail(h, status, "pressure residual %.3e above tol %.3e after %d sweeps", r,
                    h->p.tol, k);
    return LBM2P_OK;
}

// One physical step.  Its inputs (f buffer cur_f, g buffer cur_g, the current R, 1/tau_f and
// P^{n-1}) are only read; the step writes the other buffers and makes them current when it
// ends.  A step whose pressure residual is not a number (ENONFINITE) runs no saturation update
// and changes no current buffer: the state is as before the step.
lbm2p_status one_step(lbm2p *h, int replay, lbm2p_step_stats *stats)
{
    cudaStream_t st = (cudaStream_t)h->stream;
    auto fill = [&](int k, lbm2p_status ps, double r, float sw_ms, float step_ms) {
        if (stats) {
            stats->sub_iters = k;
            stats->status = ps;
            stats->residual = r;
            stats->sweep_ms = sw_ms;
            stats->step_ms = step_ms;
        }
    };
    auto advance = [&](int pout) {
        h->cur_f = pout;
        h->cur_g = 1 - h->cur_g;
        h->cur_r = 1 - h->cur_r;
    };
    if (replay < 0 && h->graph_ok) {
        cudaGraphExec_t x;
        lbm2p_status e = step_graph(h, h->cur_f, h->cur_g, &x);
        if (e != LBM2P_OK)
            return e;
        if (h->timing)
            CUDA_TRY(h, cudaEventRecord(h->ev_step0, st));
        CUDA_TRY(h, cudaGraphLaunch(x, st));
        if (h->timing)
            CUDA_TRY(h, cudaEventRecord(h->ev_step1, st));
        int k = 0;
        double r = std::nan("");
        float sw_ms = -1.0f, step_ms = -1.0f;
        if ((e = read_loop(h, &k, &r, &sw_ms)) != LBM2P_OK)
            return e;
        const bool finite = !std::isnan(r);
        // refresh and the finiteness test; saturation and rebase when the step goes on
        h->launches += finite ? 4 : 2;
        if (h->timing)
            CUDA_TRY(h, cudaEventElapsedTime(&step_ms, h->ev_step0, h->ev_step1));
        lbm2p_status ps = loop_status(h, k, r);
        if (finite)
            advance(fnext(h->cur_f, 2));
        fill(k, ps, r, sw_ms, step_ms);
        return ps;
    }
    if (h->timing)
        CUDA_TRY(h, cudaEventRecord(h->ev_step0, st));
    // a1: stream g, S^n, tau_f (and the warm start) into the work buffers
    lbm2p_launch::refresh(refresh_args(h, h->cur_g, false), h->grid, h->stream);
    LAUNCHED(h, "refresh");
    // a2/a3: pressure sub-iteration
    int k = 0, pout = h->cur_f;
    double r = std::nan("");
    float sw_ms = -1.0f;
    lbm2p_status ps = pressure_solve(h, replay, true, &k, &r, &sw_ms, &pout);
    if (ps != LBM2P_OK && ps != LBM2P_ENOTCONVERGED) {
        fill(k, ps, r, sw_ms, -1.0f);
        return ps;
    }
    // a4/a5: grad P and the saturation update
    lbm2p_launch::saturation(saturation_args(h, pout, h->cur_g, true), h->grid, h->stream);
    LAUNCHED(h, "saturation");
    lbm2p_launch::rebase(rebase_args(h, pout, true), h->grid, h->stream);
    LAUNCHED(h, "rebase");
    advance(pout);
    float step_ms = -1.0f;
    if (h->timing) {
        CUDA_TRY(h, cudaEventRecord(h->ev_step1, st));
        CUDA_TRY(h, cudaEventSynchronize(h->ev_step1));
        CUDA_TRY(h, cudaEventElapsedTime(&step_ms, h->ev_step0, h->ev_step1));
    }
    fill(k, ps, r, sw_ms, step_ms);
    return ps;
}

lbm2p_status check_params(const lbm2p_params *p, const lbm2p_inputs *in)
{
    if (!p || !in)
        return fail(nullptr, LBM2P_EINVAL, "params and inputs are required");
    if (p->nx < 1 || p->ny < 1)
        return fail(nullptr, LBM2P_EINVAL, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    long long pitch = ((long long)p->nx + 31) / 32 * 32;
    if (pitch * p->ny >= (1LL << 31) - 1024)
        return fail(nullptr, LBM2P_EINVAL, "lattice %d x %d exceeds the 2^31 plane limit", p->nx, p->ny);
    if (!(p->dx > 0) || !(p->dt > 0) || !std::isfinite(p->dx) || !std::isfinite(p->dt))
        return fail(nullptr, LBM2P_EINVAL, "dx and dt must be positive");
    if (!(p->phi > 0) || !(p->beta > 0))
        return fail(nullptr, LBM2P_EINVAL, "phi and beta must be positive");
    if (!(p->D_s > 0))
        return fail(nullptr, LBM2P_EINVAL, "D_s must be positive (tau_g > 1/2)");
    if (p->warm_start != 0 && p->warm_start != 1)
        return fail(nullptr, LBM2P_EINVAL, "warm_start must be 0 or 1");
    if (p->sat_lattice != 9 && p->sat_lattice != 5)
        return fail(nullptr, LBM2P_EINVAL, "sat_lattice must be 9 or 5 (got %d)", p->sat_lattice);
    if (!(p->D_c >= 0) || !std::isfinite(p->D_c))
        return fail(nullptr, LBM2P_EINVAL, "D_c must be finite and >= 0");
    if (p->mobility == LBM2P_MOB_QUADRATIC) {
        if (!(p->mu_w > 0) || !(p->mu_n > 0))
            return fail(nullptr, LBM2P_EINVAL, "quadratic mobility needs mu_w, mu_n > 0");
    } else if (p->mobility == LBM2P_MOB_DECOUPLED) {
        if (!(p->mu_w > 0))
            return fail(nullptr, LBM2P_EINVAL, "decoupled mobility needs mu_w > 0");
    } else if (p->mobility != LBM2P_MOB_RATIONAL) {
        return fail(nullptr, LBM2P_EINVAL, "unknown mobility law %d", p->mobility);
    }
    if (p->tau_mode == LBM2P_TAU_REFERENCE) {
        if (!(p->tau_p > 0.5))
            return fail(nullptr, LBM2P_EINVAL, "tau_p must exceed 1/2");
    } else if (p->tau_mode != LBM2P_TAU_PHYSICAL_DT) {
        return fail(nullptr, LBM2P_EINVAL, "unknown tau mode %d", p->tau_mode);
    }
    if (!(p->tol >= 0) || p->max_sub_iters < 1 || p->check_every < 1)
        return fail(nullptr, LBM2P_EINVAL, "need tol >= 0, max_sub_iters >= 1, check_every >= 1");
    for (int s = 0; s < 4; ++s)
        if (p->bc[s] < 0 || p->bc[s] > 2)
            return fail(nullptr, LBM2P_EINVAL, "unknown wall kind %d on side %d", p->bc[s], s);
    if ((p->bc[0] == LBM2P_BC_PERIODIC) != (p->bc[1] == LBM2P_BC_PERIODIC) ||
        (p->bc[2] == LBM2P_BC_PERIODIC) != (p->bc[3] == LBM2P_BC_PERIODIC))
        return fail(nullptr, LBM2P_EINVAL, "a periodic side must be paired with its opposite");
    if ((p->bc[0] == LBM2P_BC_DIRICHLET || p->bc[1] == LBM2P_BC_DIRICHLET) && p->nx < 3)
        return fail(nullptr, LBM2P_EINVAL, "Dirichlet x-sides need nx >= 3");
    if ((p->bc[2] == LBM2P_BC_DIRICHLET || p->bc[3] == LBM2P_BC_DIRICHLET) && p->ny < 3)
        return fail(nullptr, LBM2P_EINVAL, "Dirichlet y-sides need ny >= 3");
    if (p->fuse_sweeps != 0 && p->fuse_sweeps != 1 && p->fuse_sweeps != 2 && p->fuse_sweeps != 4)
        return fail(nullptr, LBM2P_EINVAL, "fuse_sweeps must be 0, 1, 2 or 4");
    if (p->sweep_kernel < LBM2P_SWEEP_AUTO || p->sweep_kernel > LBM2P_SWEEP_ROWS)
        return fail(nullptr, LBM2P_EINVAL, "sweep_kernel must be an lbm2p_sweep_kernel value");
    if (p->storage != LBM2P_STORE_FP32 && p->storage != LBM2P_STORE_FP16_DEV)
        return fail(nullptr, LBM2P_EINVAL, "unknown storage %d", p->storage);
    if (!in->K || !in->S0)
        return fail(nullptr, LBM2P_EINVAL, "K and S0 are required");
    if (in->n_wells < 0 || in->n_wells > LBM2P_MAX_WELLS || (in->n_wells > 0 && !in->wells))
        return fail(nullptr, LBM2P_EINVAL, "0..%d wells supported", LBM2P_MAX_WELLS);
    for (int m = 0; m < in->n_wells; ++m) {
        const lbm2p_well &w = in->wells[m];
        if (w.i < 0 || w.i >= p->nx || w.j < 0 || w.j >= p->ny || !(w.q >= 0) || !std::isfinite(w.q))
            return fail(nullptr, LBM2P_EINVAL, "well %d out of range or negative rate", m);
    }
    const long long n = (long long)p->nx * p->ny;
    for (long long a = 0; a < n; ++a) {
        if (!(in->K[a] > 0) || !std::isfinite(in->K[a]))
            return fail(nullptr, LBM2P_EINVAL, "K must be positive and finite (node %lld)", a);
        if (!std::isfinite(in->S0[a]))
            return fail(nullptr, LBM2P_EINVAL, "S0 must be finite (node %lld)", a);
    }
    if (in->init_replay && *in->init_replay < 0)
        return fail(nullptr, LBM2P_EINVAL, "init_replay must be >= 0");
    return LBM2P_OK;
}

// Pick how the pressure sweeps run on this lattice by timing every candidate: the single-
// sweep kernels (the staged-rows one over strip widths and rows per block), and (when
// allowed) T = 2 and 4 fused sweeps over each tile shape (W columns, H rows).  A requested
// single-sweep kernel is the only one timed; requested fused sweeps win over single ones.
// Each candidate runs once untimed, then the best of two timed groups of reps launches
// counts.  Runs on the zeroed buffers before initialisation; they are zeroed again after.
// a fused form must take at most this fraction of the best single sweep's time per sweep
constexpr float kFusedMargin = 0.95f;

lbm2p_status autotune_sweeps(lbm2p *h)
{
    cudaStream_t st = (cudaStream_t)h->stream;
    for (auto &a : h->allocs)
        CUDA_TRY(h, cudaMemsetAsync(a.ptr, 0, a.bytes, st));
    int dev = 0, sms = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    lbm2p_status status = LBM2P_OK;
    const int reps = 6;
    // per-launch time of a candidate: best of two groups of reps launches after one warm-up
    auto timed = [&](auto launch, float *ms) -> bool {
        launch(0);
        float best_ms = 1e30f;
        for (int trial = 0; trial < 2; ++trial) {
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < reps; ++rep)
                launch(rep + 1);
            cudaEventRecord(e1, st);
            cudaError_t le = cudaEventSynchronize(e1);
            if (le != cudaSuccess) {
                status = fail(h, LBM2P_ECUDA, "sweep timing failed: %s", cudaGetErrorString(le));
                return false;
            }
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            best_ms = t < best_ms ? t : best_ms;
        }
        *ms = best_ms / reps;
        return true;
    };
    const int forced = h->p.sweep_kernel;                  // 0: any single-sweep kernel
    auto allowed = [&](int kind) { return forced == LBM2P_SWEEP_AUTO || forced == kind + 1; };
    const bool fused_only = h->p.fuse_sweeps == 2 || h->p.fuse_sweeps == 4;
    float best = 1e30f;                                    // per-sweep time of the choice
    // a fused form replaces single sweeps only when it is clearly faster: in the timed solve
    // loop the forms come out closer than these timings say (1024^2 five-spot: the two-sweep
    // direct form estimated 8 % ahead here with a 16-sweep check period and 3.5 % ahead in the
    // loop; 8 % ahead with an 8-sweep period and about even in the loop)
    float single_best = 1e30f;
    auto fused_wins = [&](float per) {
        return h->tb_T > 1 ? per < best : (per < best && per < kFusedMargin * single_best);
    };
    h->autotune_log.clear();
    auto note = [&](const char *what, int a1, int a2, int a3, int a4, float us) {
        char line[160];
        snprintf(line, sizeof line, "%s %d %d %d %d %.3f\n", what, a1, a2, a3, a4, us);
        h->autotune_log += line;
    };
    // what a candidate costs per sweep inside the solve loop: a check period of check_every
    // sweeps runs (launches - 1) plain launches and one that also sums the residual
    const int m_chk = h->p.check_every;
    auto in_loop = [&](float plain, float check, int T) {
        const int nl = m_chk / T > 0 ? m_chk / T : 1;
        return ((float)(nl - 1) * plain + check) / (float)(nl * T);
    };
    // the checking launch's time, when its residual partials fit the scratch array
    auto timed_check = [&](auto launch, long long parts, float plain, float *ms) -> bool {
        *ms = plain;
        if (parts > h->partials_cap)
            return true;
        return timed(launch, ms);
    };
    h->tb_T = 0;
    h->sweep_kind = forced == LBM2P_SWEEP_AUTO ? 0 : forced - 1;
    if (!fused_only || forced != LBM2P_SWEEP_AUTO) {
        // grid-stride kernels: resident blocks per SM from the occupancy limit down to half
        // of it (fewer, fuller rounds of row tiles per block can beat a full machine)
        for (int kind = 0; kind < 2; ++kind) {
            if (!allowed(kind))
                continue;
            const int maxb = lbm2p_launch::max_blocks_per_sm_pressure(false, kind);
            float best_kind = 1e30f;
            int best_grid = h->grid_k[kind], last_grid = -1;
            for (int b = maxb; b >= 1 && 2 * b >= maxb; --b) {
                long long want = (long long)sms * b;
                want = want < h->geom.ntiles ? want : h->geom.ntiles;
                const int grid = (int)(want > 0 ? want : 1);
                if (grid == last_grid)
                    continue;
                last_grid = grid;
                float ms = 0.0f, mc = 0.0f;
                if (!timed([&](int k) {
                        PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                        lbm2p_launch::pressure_sweep(a, false, false, grid, h->stream, kind);
                    }, &ms))
                    goto done;
                if (!timed_check([&](int k) {
                        PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                        lbm2p_launch::pressure_sweep(a, true, false, h->grid_check_k[kind], h->stream,
                                                     kind);
                    }, h->grid_check_k[kind], ms, &mc))
                    goto done;
                ms = in_loop(ms, mc, 1);
                note(kind == 0 ? "single_vec4" : "single_scalar", grid, 0, 0, 0, ms * 1e3f);
                if (ms < best_kind) {
                    best_kind = ms;
                    best_grid = grid;
                }
            }
            h->grid_k[kind] = best_grid;
            if (best_kind < best) {
                best = best_kind;
                h->sweep_kind = kind;
            }
        }
        // the staged-rows kernel: strip width, ring slots, and rows per block giving 1 to 16
        // blocks per resident block slot
        const int shapes[3][2] = {{128, 8}, {256, 6}, {256, 8}};
        float best_rows = 1e30f;
        int rows_shape[4] = {0, 0, 0, 0};                  // width, slots, H, grid
        for (const auto &sh : shapes) {
            if (!allowed(2))
                break;
            const int width = sh[0], slots = sh[1];
            if (lbm2p_launch::rows_prepare(width, slots) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            const int per_sm = lbm2p_launch::rows_blocks_per_sm(width, slots, h->Fp != nullptr);
            if (per_sm < 1)
                continue;
            const int strips = (h->nx + width - 1) / width;
            int last_H = -1;
            for (int mult : {1, 2, 4, 8, 16}) {
                const long long want = (long long)sms * per_sm * mult;
                long long chunks = (want + strips - 1) / strips;
                chunks = chunks < 1 ? 1 : chunks;
                const int H = (int)((h->ny + chunks - 1) / chunks);
                if (H == last_H)
                    continue;
                last_H = H;
                const int grid = (int)lbm2p_launch::rows_grid(width, H, h->nx, h->ny);
                float ms = 0.0f, mc = 0.0f;
                if (!timed([&](int k) {
                        PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                        lbm2p_launch::pressure_sweep_rows(a, false, false, width, slots, H, grid,
                                                          h->stream);
                    }, &ms))
                    goto done;
                if (!timed_check([&](int k) {
                        PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                        lbm2p_launch::pressure_sweep_rows(a, true, false, width, slots, H, grid,
                                                          h->stream);
                    }, grid, ms, &mc))
                    goto done;
                ms = in_loop(ms, mc, 1);
                note("single_rows", width, slots, H, grid, ms * 1e3f);
                if (ms < best_rows) {
                    best_rows = ms;
                    rows_shape[0] = width;
                    rows_shape[1] = slots;
                    rows_shape[2] = H;
                    rows_shape[3] = grid;
                }
            }
        }
        if (rows_shape[0] > 0 && (best_rows < best || forced == LBM2P_SWEEP_ROWS)) {
            best = best_rows;
            h->sweep_kind = 2;
        }
        if (rows_shape[0] > 0) {
            h->rows_w = rows_shape[0];
            h->rows_slots = rows_shape[1];
            h->rows_H = rows_shape[2];
            h->rows_grid = rows_shape[3];
        }
        if (forced == LBM2P_SWEEP_ROWS && rows_shape[0] == 0) {
            status = fail(h, LBM2P_ENOTIMPL, "the staged-rows sweep kernel cannot run here");
            goto done;
        }
    }
    if (fused_only)
        best = 1e30f;
    single_best = best;
    if (h->p.fuse_sweeps != 1) {
        bool walls = true;
        for (int sd = 0; sd < 4; ++sd)
            walls = walls && h->p.bc[sd] != LBM2P_BC_PERIODIC;
        // fuse_sweeps 2 with the ROWS kernel pinned asks for the staged-rows two-sweep kernel,
        // with the SCALAR kernel pinned for the direct-load one
        const bool rows2_only = walls && h->p.fuse_sweeps == 2 && forced == LBM2P_SWEEP_ROWS;
        const bool direct_only = walls && h->p.fuse_sweeps == 2 && forced == LBM2P_SWEEP_SCALAR;
        for (int T : {2, 4}) {
            if ((h->p.fuse_sweeps != 0 && h->p.fuse_sweeps != T) || rows2_only || direct_only)
                continue;
            for (int W : {128, 64, 32}) {
                cudaError_t ce = lbm2p_launch::tb_prepare(T, W);
                if (ce != cudaSuccess || lbm2p_launch::tb_blocks_per_sm(T, W) < 1) {
                    cudaGetLastError();
                    continue;
                }
                for (int H : {64, 32, 16, 8}) {
                    const long long blocks = lbm2p_launch::tb_grid(T, W, H, h->nx, h->ny);
                    if (blocks > (1LL << 30))
                        continue;
                    float ms = 0.0f, mc = 0.0f;
                    if (!timed([&](int k) {
                            PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                            lbm2p_launch::pressure_sweeps_fused(a, T, W, H, false, (int)blocks,
                                                                h->stream);
                        }, &ms))
                        goto done;
                    if (!timed_check([&](int k) {
                            PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                            lbm2p_launch::pressure_sweeps_fused(a, T, W, H, true, (int)blocks,
                                                                h->stream);
                        }, blocks, ms, &mc))
                        goto done;
                    const float per = in_loop(ms, mc, T);
                    note("fused", T, W, H, (int)blocks, per * 1e3f);
                    if (fused_wins(per)) {
                        best = per;
                        h->tb_T = T;
                        h->tb_kind = 0;
                        h->tb_W = W;
                        h->tb_H = H;
                        h->tb_grid = (int)blocks;
                    }
                }
            }
        }
        // two sweeps per launch on rows staged by bulk copies (lattices with walls on every
        // side): consumer warps x ring slots, and output rows per block
        // two sweeps per launch with direct loads (for lattices whose populations stay in L2)
        if (walls && (h->p.fuse_sweeps == 0 || h->p.fuse_sweeps == 2) &&
            (forced == LBM2P_SWEEP_AUTO || forced == LBM2P_SWEEP_SCALAR)) {
            for (int cw : {4, 8}) {
                int last_H = -1;
                for (int H : {2, 4, 8, 16, 32}) {
                    const int Hc = H < h->ny ? H : h->ny;
                    if (Hc == last_H)
                        continue;
                    last_H = Hc;
                    const long long blocks = lbm2p_launch::pair_direct_grid(cw, Hc, h->nx, h->ny);
                    if (blocks > (1LL << 30))
                        continue;
                    float ms = 0.0f, mc = 0.0f;
                    if (!timed([&](int k) {
                            PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                            lbm2p_launch::pressure_sweeps_pair_direct(a, false, cw, Hc, (int)blocks,
                                                                      h->stream);
                        }, &ms))
                        goto done;
                    if (!timed_check([&](int k) {
                            PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                            lbm2p_launch::pressure_sweeps_pair_direct(a, true, cw, Hc, (int)blocks,
                                                                      h->stream);
                        }, blocks, ms, &mc))
                        goto done;
                    const float per = in_loop(ms, mc, 2);
                    note("fused_direct", cw, 0, Hc, (int)blocks, per * 1e3f);
                    if (fused_wins(per) || (direct_only && h->tb_kind != 2)) {
                        best = per;
                        h->tb_T = 2;
                        h->tb_kind = 2;
                        h->tb_W = 30 * cw;
                        h->tb_slots = 0;
                        h->tb_H = Hc;
                        h->tb_grid = (int)blocks;
                    }
                }
            }
        }
        if (walls && !direct_only && (h->p.fuse_sweeps == 0 || h->p.fuse_sweeps == 2) &&
            (forced == LBM2P_SWEEP_AUTO || forced == LBM2P_SWEEP_ROWS)) {
            const int shapes2[5][2] = {{4, 6}, {4, 8}, {8, 4}, {8, 6}, {4, 6 + lbm2p_launch::kRows2Dense}};
            for (const auto &sh : shapes2) {
                const int cw = sh[0], slots = sh[1];
                if (lbm2p_launch::rows2_prepare(cw, slots) != cudaSuccess ||
                    lbm2p_launch::rows2_blocks_per_sm(cw, slots, h->Fp != nullptr) < 1) {
                    cudaGetLastError();
                    continue;
                }
                int last_H = -1;
                for (int H : {16, 32, 64, 128}) {
                    const int Hc = H < h->ny ? H : h->ny;
                    if (Hc == last_H)
                        continue;
                    last_H = Hc;
                    const long long blocks = lbm2p_launch::rows2_grid(cw, Hc, h->nx, h->ny);
                    if (blocks > (1LL << 30))
                        continue;
                    float ms = 0.0f, mc = 0.0f;
                    if (!timed([&](int k) {
                            PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                            lbm2p_launch::pressure_sweeps_rows2(a, false, cw, slots, Hc,
                                                                (int)blocks, h->stream);
                        }, &ms))
                        goto done;
                    if (!timed_check([&](int k) {
                            PressureArgs a = pressure_args(h, k % 2, 1 - k % 2, false);
                            lbm2p_launch::pressure_sweeps_rows2(a, true, cw, slots, Hc,
                                                                (int)blocks, h->stream);
                        }, blocks, ms, &mc))
                        goto done;
                    const float per = in_loop(ms, mc, 2);
                    note("fused_rows", cw, slots, Hc, (int)blocks, per * 1e3f);
                    if (fused_wins(per)) {
                        best = per;
                        h->tb_T = 2;
                        h->tb_kind = 1;
                        h->tb_W = lbm2p_launch::rows2_width(cw);
                        h->tb_slots = slots;
                        h->tb_H = Hc;
                        h->tb_grid = (int)blocks;
                    }
                }
            }
        }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != LBM2P_OK)
        return status;
    CUDA_TRY(h, cudaGetLastError());
    for (auto &a : h->allocs)
        CUDA_TRY(h, cudaMemsetAsync(a.ptr, 0, a.bytes, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return LBM2P_OK;
}

// FP16 storage: time the one-node-per-thread FP16 sweep and the FP16 staged-rows sweep over
// its shapes on this lattice (zeroed buffers) and keep the fastest
lbm2p_status autotune_h(lbm2p *h, int sms)
{
    cudaStream_t st = (cudaStream_t)h->stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    auto args = [&](int k) {
        HalfSweepArgs a{};
        for (int i = 0; i < 8; ++i) {
            a.nin[i] = h->hbuf[k & 1][i];
            a.nout[i] = h->hbuf[1 - (k & 1)][i];
        }
        a.Rin = h->Rh[k & 1];
        a.Rout = h->Rh[1 - (k & 1)];
        a.inv_tau = itau_of(h, false);
        a.Fp = h->Fp;
        a.partials = h->partials;
        a.shift = h->shift;
        a.scale = h->hscale;
        a.scale_out = h->hscale;
        for (int s = 0; s < 4; ++s)
            a.Pb[s] = h->Pb[s];
        a.g = h->geom;
        a.w = h->wells;
        return a;
    };
    lbm2p_status status = LBM2P_OK;
    const int reps = 6;
    auto timed = [&](auto launch, float *ms) -> bool {
        launch(0);
        float best_ms = 1e30f;
        for (int trial = 0; trial < 2; ++trial) {
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < reps; ++rep)
                launch(rep + 1);
            cudaEventRecord(e1, st);
            cudaError_t le = cudaEventSynchronize(e1);
            if (le != cudaSuccess) {
                status = fail(h, LBM2P_ECUDA, "FP16 sweep timing failed: %s", cudaGetErrorString(le));
                return false;
            }
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            best_ms = t < best_ms ? t : best_ms;
        }
        *ms = best_ms / reps;
        return true;
    };
    char line[160];
    float best = 1e30f;
    const bool rows_only = h->p.sweep_kernel == LBM2P_SWEEP_ROWS;
    const bool no_rows = h->p.sweep_kernel == LBM2P_SWEEP_SCALAR || h->p.sweep_kernel == LBM2P_SWEEP_VEC4;
    h->h16_kind = 0;
    {
        float ms = 0.0f;
        if (!timed([&](int k) { lbm2p_launch::pressure_sweep_h(args(k), false, h->grid_h, h->stream); },
                   &ms))
            goto done;
        snprintf(line, sizeof line, "fp16_scalar %d 0 0 0 %.3f\n", h->grid_h, ms * 1e3f);
        h->autotune_log += line;
        best = rows_only ? 1e30f : ms;
    }
    if (!no_rows) {
        const int shapes[3][2] = {{128, 8}, {256, 6}, {256, 8}};
        for (const auto &sh : shapes) {
            const int width = sh[0], slots = sh[1];
            if (lbm2p_launch::rows_h_prepare(width, slots) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            const int per_sm = lbm2p_launch::rows_h_blocks_per_sm(width, slots, h->Fp != nullptr);
            if (per_sm < 1)
                continue;
            const int strips = (h->nx + width - 1) / width;
            int last_H = -1;
            for (int mult : {1, 2, 4, 8, 16}) {
                long long chunks = ((long long)sms * per_sm * mult + strips - 1) / strips;
                chunks = chunks < 1 ? 1 : chunks;
                const int H = (int)((h->ny + chunks - 1) / chunks);
                if (H == last_H)
                    continue;
                last_H = H;
                const int grid = (int)lbm2p_launch::rows_grid(width, H, h->nx, h->ny);
                float ms = 0.0f;
                if (!timed([&](int k) {
                        lbm2p_launch::pressure_sweep_rows_h(args(k), false, width, slots, H, grid,
                                                            h->stream);
                    }, &ms))
                    goto done;
                snprintf(line, sizeof line, "fp16_rows %d %d %d %d %.3f\n", width, slots, H, grid,
                         ms * 1e3f);
                h->autotune_log += line;
                if (ms < best) {
                    best = ms;
                    h->h16_kind = 1;
                    h->h16_w = width;
                    h->h16_slots = slots;
                    h->h16_H = H;
                    h->h16_grid = grid;
                }
            }
        }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != LBM2P_OK)
        return status;
    CUDA_TRY(h, cudaGetLastError());
    for (auto &a : h->allocs)
        CUDA_TRY(h, cudaMemsetAsync(a.ptr, 0, a.bytes, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return LBM2P_OK;
}

lbm2p_status build(lbm2p *h, const lbm2p_inputs *in, lbm2p_step_stats *init_stats)
{
    const lbm2p_params &p = h->p;
    h->nx = p.nx;
    h->ny = p.ny;
    h->pitch = (p.nx + 31) / 32 * 32;
    h->plane = (long long)h->pitch * p.ny;
    h->nnodes = (long long)p.nx * p.ny;
    h->stream = p.stream;
    Geom &g = h->geom;
    g.nx = p.nx;
    g.ny = p.ny;
    g.pitch = h->pitch;
    g.tiles_x = (p.nx + kBlock - 1) / kBlock;
    g.ntiles = g.tiles_x * p.ny;
    for (int s = 0; s < 4; ++s)
        g.bc[s] = p.bc[s];

    // pseudo-time scale s and the relaxation times (Eq. 3-11)
    h->tau_g = 0.5 + 3.0 * p.D_s * p.dt / (p.beta * p.dx * p.dx);
    if (p.tau_mode == LBM2P_TAU_REFERENCE) {
        double D = p.D_ref;
        if (!(D > 0)) {
            double acc = 0.0;
            for (long long a = 0; a < h->nnodes; ++a)
                acc += std::log(in->K[a] * lambda_t_host(p, in->S0[a]));
            D = std::exp(acc / (double)h->nnodes);
        }
        if (!(D > 0) || !std::isfinite(D))
            return fail(h, LBM2P_EINVAL, "reference diffusivity is not positive");
        h->D_ref = D;
        h->s = (p.tau_p - 0.5) / (3.0 * D);
    } else {
        h->s = p.dt / (p.dx * p.dx);
    }
    Model &m = h->model;
    m.mobility = p.mobility;
    m.inv_mu_w = (float)(1.0 / p.mu_w);
    m.inv_mu_n = p.mobility == LBM2P_MOB_QUADRATIC ? (float)(1.0 / p.mu_n) : 0.0f;
    m.phi = (float)p.phi;
    m.inv_phi = (float)(1.0 / p.phi);
    m.s3 = (float)(3.0 * h->s);
    m.fs_scale = (float)p.dt;
    m.inv_tau_g = (float)(1.0 / h->tau_g);
    m.src_g = (float)(1.0 - 0.5 / h->tau_g);
    m.gam_c = (float)(3.0 * p.dt / (p.dx * p.dx));
    m.inv_dx = (float)(1.0 / p.dx);
    // Eq. 3-4: g_i^eq / S = w_i [phi + (beta - phi)(|c_i|^2 - 2 c_s^2) / (2 c_s^2)], c_s^2 = 1/3
    m.qs = p.sat_lattice;
    for (int i = 0; i < 9; ++i) {
        const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double c2 = (double)(cx(i) * cx(i) + cy(i) * cy(i));
        m.Gam[i] = (float)(w * (p.phi + (p.beta - p.phi) * (c2 - 2.0 / 3.0) / (2.0 / 3.0)));
        m.wg[i] = (float)w;
    }
    if (p.sat_lattice == 5) {
        // D2Q5 (Remark V): weights 1/3 and 1/6; Eq. 3-4b: g_0^eq / S = (w_0 - 1) beta + phi,
        // g_i^eq / S = w_i beta
        for (int i = 0; i < 9; ++i) {
            const double w = i == 0 ? 1.0 / 3.0 : (i <= 4 ? 1.0 / 6.0 : 0.0);
            m.wg[i] = (float)w;
            m.Gam[i] = (float)(i == 0 ? (w - 1.0) * p.beta + p.phi : w * p.beta);
        }
    }
    m.var_ds = p.D_c != 0.0 ? 1 : 0;
    m.ds_a0 = (float)(3.0 * p.D_s * p.dt / (p.beta * p.dx * p.dx));
    m.ds_a1 = (float)(3.0 * p.D_c * p.dt / (p.beta * p.dx * p.dx));
    Wells &w = h->wells;
    w.n = in->n_wells;
    for (int k = 0; k < in->n_wells; ++k) {
        const lbm2p_well &wl = in->wells[k];
        w.idx[k] = wl.j * h->pitch + wl.i;
        w.producer[k] = wl.is_producer ? 1 : 0;
        // F~_p = s dx^2 * (+-q / dx^2);  dt F_s magnitude = dt q / dx^2
        w.fp[k] = (float)(wl.is_producer ? -h->s * wl.q : h->s * wl.q);
        w.qs[k] = (float)(p.dt * wl.q / (p.dx * p.dx));
    }

    // device memory
    int dev = 0, sms = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // grids: the resident-block capacity of the GPU (multiples of the SM count), capped by
    // the number of row tiles of the widest kernel work item
    auto cap_grid = [&](long long blocks) {
        const long long tiles = (long long)g.ntiles;
        if (blocks > tiles)
            blocks = tiles;
        return (int)(blocks > 0 ? blocks : 1);
    };
    for (int kind = 0; kind < 2; ++kind) {
        h->grid_cap_k[kind] = cap_grid((long long)sms * lbm2p_launch::max_blocks_per_sm_pressure(false, kind));
        h->grid_k[kind] = h->grid_cap_k[kind];
        h->grid_check_k[kind] = cap_grid((long long)sms * lbm2p_launch::max_blocks_per_sm_pressure(true, kind));
    }
    h->sweep_kind = 0;
    h->grid = h->grid_k[0];
    h->grid_check = h->grid_check_k[0];
    const size_t pb = (size_t)h->plane * sizeof(float);
    auto plane_alloc = [&](float **dst) -> bool {
        *dst = (float *)dev_alloc(h, pb);
        return *dst != nullptr;
    };
    bool ok = true;
    for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 8; ++i)
            ok = ok && plane_alloc(&h->fbuf[b][i]);
    for (int b = 0; b < 2; ++b) {
        for (int i = 0; i < 9; ++i)
            ok = ok && plane_alloc(&h->gbuf[b][i]);
    }
    for (int b = 0; b < 2; ++b) {
        ok = ok && plane_alloc(&h->inv_taub[b]) && plane_alloc(&h->Rb[b]);
        if (p.warm_start)
            ok = ok && plane_alloc(&h->Pstepb[b]);
    }
    ok = ok && plane_alloc(&h->K) && plane_alloc(&h->S) && plane_alloc(&h->Pio) &&
         plane_alloc(&h->tmp);
    if (in->Fp)
        ok = ok && plane_alloc(&h->Fp);
    if (in->Fs)
        ok = ok && plane_alloc(&h->Fs);
    for (int s = 0; s < 4; ++s) {
        if (p.bc[s] == LBM2P_BC_DIRICHLET) {
            h->Pb[s] = (float *)dev_alloc(h, (size_t)trace_len(h, s) * sizeof(float));
            h->Sb[s] = (float *)dev_alloc(h, (size_t)trace_len(h, s) * sizeof(float));
            ok = ok && h->Pb[s] && h->Sb[s];
        }
    }
    h->fp16 = p.storage == LBM2P_STORE_FP16_DEV;
    if (h->fp16) {
        // FP16 copies of the populations and the per-sweep node pressures of a solve
        for (int b = 0; b < 2; ++b) {
            for (int i = 0; i < 8; ++i) {
                h->hbuf[b][i] = (__half *)dev_alloc(h, (size_t)h->plane * sizeof(__half));
                ok = ok && h->hbuf[b][i];
            }
            ok = ok && plane_alloc(&h->Rh[b]);
        }
        h->hscale = (float *)dev_alloc(h, 64);
        ok = ok && h->hscale;
        CUDA_TRY(h, cudaMallocHost((void **)&h->hscale_host, 4 * sizeof(float)));
        h->grid_h = cap_grid((long long)sms * lbm2p_launch::max_blocks_per_sm_pressure_h());
    }
    if (!ok)
        return fail(h, LBM2P_ENOMEM, "device allocation of %.1f MiB failed",
                    (double)pb * 45 / (1 << 20));
    // which single-sweep kernel, single or fused sweeps, and the fused tile shape: timed
    // on this lattice (within what fuse_sweeps allows); FP16 storage has one sweep kernel
    if (!h->fp16) {
        // the timing of each candidate's checking launch needs residual partials and shift
        // constants: a partials array sized for the finest candidate grid (a block owns at
        // least 128 nodes), kept as the handle's own when it is large enough
        h->partials_cap = h->nnodes / 128 + 4096;
        h->partials = (double *)dev_alloc(h, (size_t)h->partials_cap * 4 * sizeof(double));
        h->shift = (float *)dev_alloc(h, 64);
        if (!h->partials || !h->shift)
            return fail(h, LBM2P_ENOMEM, "device allocation of the residual partials failed");
        lbm2p_status e = autotune_sweeps(h);
        if (e != LBM2P_OK)
            return e;
    } else {
        h->sweep_kind = 1;
        h->tb_T = 0;
        lbm2p_status e = autotune_h(h, sms);
        if (e != LBM2P_OK)
            return e;
    }
    // grid-stride lattice kernels keep the one-node-per-thread capacity when the staged
    // sweep is chosen
    h->grid = h->grid_cap_k[h->sweep_kind < 2 ? h->sweep_kind : 1];
    h->grid_sweep = h->grid_k[h->sweep_kind < 2 ? h->sweep_kind : 1];
    h->grid_check = h->grid_check_k[h->sweep_kind < 2 ? h->sweep_kind : 1];
    {
        int np = h->tb_grid > h->rows_grid ? h->tb_grid : h->rows_grid;
        np = np > h->grid_h ? np : h->grid_h;
        np = np > h->h16_grid ? np : h->h16_grid;
        for (int kind = 0; kind < 2; ++kind) {
            np = np > h->grid_k[kind] ? np : h->grid_k[kind];
            np = np > h->grid_check_k[kind] ? np : h->grid_check_k[kind];
        }
        if (!h->partials || np > h->partials_cap) {
            h->partials = (double *)dev_alloc(h, (size_t)np * 4 * sizeof(double));
            h->partials_cap = np;
        }
    }
    h->mean = (double *)dev_alloc(h, 64);
    if (!h->shift)
        h->shift = (float *)dev_alloc(h, 64);
    h->res = (ResidualOut *)dev_alloc(h, sizeof(ResidualOut));
    h->ctl = (LoopCtl *)dev_alloc(h, sizeof(LoopCtl));
    h->stage = (float *)dev_alloc(h, (size_t)h->nnodes * sizeof(float) * 4);
    ok = ok && h->partials && h->mean && h->shift && h->res && h->ctl && h->stage;
    if (!ok)
        return fail(h, LBM2P_ENOMEM, "device allocation of %.1f MiB failed",
                    (double)pb * 45 / (1 << 20));
    CUDA_TRY(h, cudaMallocHost((void **)&h->res_host, sizeof(ResidualOut)));
    CUDA_TRY(h, cudaMallocHost((void **)&h->ctl_host, sizeof(LoopCtl)));
    for (cudaEvent_t *e : {&h->ev_step0, &h->ev_step1, &h->ev_sw0, &h->ev_sw1})
        CUDA_TRY(h, cudaEventCreate(e));
    cudaStream_t st = (cudaStream_t)h->stream;
    for (auto &a : h->allocs)
        CUDA_TRY(h, cudaMemsetAsync(a.ptr, 0, a.bytes, st));
    // a long solve moves R to the current P about every 1024 sweeps (at a check point);
    // FP16 sweeps move it every sweep
    h->rebase_every = h->fp16 ? 0 : p.check_every * ((1024 + p.check_every - 1) / p.check_every);
    // the loop body holds check_every sweeps and must return to the same f buffer
    h->graph_ok = !h->fp16 && p.check_every >= 2 && p.check_every % 2 == 0 &&
                  p.max_sub_iters % p.check_every == 0;
    if (h->tb_T > 1 && p.check_every % (2 * h->tb_T) != 0)
        h->tb_T_graph = 0;
    else
        h->tb_T_graph = h->tb_T;
    {
        LoopCtl c{};
        c.m = p.check_every;
        c.cap = p.max_sub_iters;
        c.every = h->rebase_every;
        c.tol = p.tol;
        c.r = 0.0;
        *h->ctl_host = c;
        CUDA_TRY(h, cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(LoopCtl), cudaMemcpyHostToDevice, st));
        CUDA_TRY(h, cudaStreamSynchronize(st));
    }

    // inputs
    lbm2p_status e;
    if ((e = upload_plane(h, h->K, in->K, 1.0)) != LBM2P_OK)
        return e;
    if (in->Fp && (e = upload_plane(h, h->Fp, in->Fp, h->s * p.dx * p.dx)) != LBM2P_OK)
        return e;
    if (in->Fs && (e = upload_plane(h, h->Fs, in->Fs, p.dt)) != LBM2P_OK)
        return e;
    for (int s = 0; s < 4; ++s) {
        if (p.bc[s] == LBM2P_BC_DIRICHLET) {
            if ((e = upload_trace(h, h->Pb[s], in->P_b[s], trace_len(h, s))) != LBM2P_OK)
                return e;
            if ((e = upload_trace(h, h->Sb[s], in->S_b[s], trace_len(h, s))) != LBM2P_OK)
                return e;
        }
    }
    // a6: f = f^eq(P0), tau_f from S0, the t = 0 pressure solve, then g(0) and its collision
    if ((e = upload_plane(h, h->tmp, in->S0, 1.0)) != LBM2P_OK)   // tmp holds S0
        return e;
    // f^+ = f^eq(P0): reference R = P0 and zero deviations (the planes are zeroed above)
    if (in->P0 && (e = upload_plane(h, R_of(h, false), in->P0, 1.0)) != LBM2P_OK)
        return e;
    h->cur_f = 0;
    h->cur_g = 0;
    h->cur_r = 0;
    lbm2p_launch::tau_from_S(itau_of(h, false), h->tmp, h->K, g, m, h->grid, h->stream);
    LAUNCHED(h, "tau from S");
    int k0 = 0;
    double r0 = std::nan("");
    float ms0 = -1.0f, solve_ms = -1.0f;
    // the t = 0 solve is timed on the device on its own (the autotuning above and the
    // uploads are outside the two events)
    CUDA_TRY(h, cudaEventRecord(h->ev_step0, st));
    int pout = h->cur_f;
    lbm2p_status ps = pressure_solve(h, in->init_replay ? *in->init_replay : -1, false, &k0, &r0,
                                     &ms0, &pout);
    h->cur_f = pout;
    if (cudaEventRecord(h->ev_step1, st) == cudaSuccess &&
        cudaEventSynchronize(h->ev_step1) == cudaSuccess)
        cudaEventElapsedTime(&solve_ms, h->ev_step0, h->ev_step1);
    if (init_stats) {
        init_stats->sub_iters = k0;
        init_stats->status = ps;
        init_stats->residual = r0;
        init_stats->sweep_ms = ms0;
        init_stats->step_ms = solve_ms;
    }
    if (ps != LBM2P_OK && ps != LBM2P_ENOTCONVERGED)
        return ps;
    InitGArgs a{};
    for (int i = 0; i < 8; ++i)
        a.fin[i] = h->fbuf[h->cur_f][i];
    a.R = R_of(h, false);
    a.Pnew = h->Pio;
    for (int i = 0; i < 9; ++i)
        a.gout[i] = h->gbuf[0][i];
    a.K = h->K;
    a.inv_tau = itau_of(h, false);
    a.Fs = h->Fs;
    a.S0 = h->tmp;
    a.S = h->S;
    for (int s = 0; s < 4; ++s) {
        a.Pb[s] = h->Pb[s];
        a.Sb[s] = h->Sb[s];
    }
    a.g = g;
    a.m = m;
    a.w = w;
    lbm2p_launch::init_g(a, h->grid, h->stream);
    LAUNCHED(h, "init g");
    lbm2p_launch::rebase(rebase_args(h, h->cur_f, false), h->grid, h->stream);
    LAUNCHED(h, "rebase");
    if (h->p.warm_start)               // no history yet: the first step extrapolates nothing
        CUDA_TRY(h, cudaMemcpyAsync(Pstep_of(h, false), R_of(h, false),
                                    (size_t)h->plane * sizeof(float), cudaMemcpyDeviceToDevice, st));
    h->cur_g = 0;
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return ps;
}

}  // namespace

namespace lbm2p_internal {
lbm2p_status set_global_error(lbm2p_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_create_error = buf;
    return st;
}
}  // namespace lbm2p_internal

extern "C" {

int lbm2p_abi_version(void) { return LBM2P_ABI_VERSION; }

void lbm2p_default_params(lbm2p_params *p)
{
    if (!p)
        return;
    std::memset(p, 0, sizeof *p);
    p->nx = p->ny = 64;
    p->dx = 1.0 / 64;
    p->dt = 4.0 * p->dx * p->dx;
    p->phi = 0.2;
    p->beta = 0.4;
    p->mobility = LBM2P_MOB_QUADRATIC;
    p->mu_w = 1.0;
    p->mu_n = 2.0;
    p->D_s = 0.01;
    p->tau_mode = LBM2P_TAU_REFERENCE;
    p->tau_p = 1.0;
    p->D_ref = 0.0;
    p->tol = 1e-8;
    p->max_sub_iters = 10000000;
    p->check_every = 8;
    p->fuse_sweeps = 0;
    p->sweep_kernel = LBM2P_SWEEP_AUTO;
    p->sat_lattice = 9;
    p->warm_start = 0;
    p->D_c = 0.0;
    for (int s = 0; s < 4; ++s)
        p->bc[s] = LBM2P_BC_NOFLUX;
    p->storage = LBM2P_STORE_FP32;
}

lbm2p_status lbm2p_create(lbm2p **out, const lbm2p_params *p, const lbm2p_inputs *in,
                          lbm2p_step_stats *init_stats)
{
    if (!out)
        return fail(nullptr, LBM2P_EINVAL, "out must not be NULL");
    *out = nullptr;
    lbm2p_status st = check_params(p, in);
    if (st != LBM2P_OK)
        return st;
    lbm2p *h = new (std::nothrow) lbm2p();
    if (!h)
        return fail(nullptr, LBM2P_ENOMEM, "host allocation failed");
    h->p = *p;
    try {
        st = build(h, in, init_stats);
    } catch (const std::bad_alloc &) {
        st = fail(h, LBM2P_ENOMEM, "host allocation failed");
    }
    if (st != LBM2P_OK && st != LBM2P_ENOTCONVERGED) {
        g_create_error = h->err;
        if (h->stream)
            cudaStreamSynchronize((cudaStream_t)h->stream);
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return st;
}

lbm2p_status lbm2p_set_sources(lbm2p *h, const double *Fp, const double *Fs)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if ((Fp && !h->Fp) || (Fs && !h->Fs))
        return fail(h, LBM2P_EINVAL, "dense sources must be given at create to be replaced");
    lbm2p_status e;
    cudaStream_t st = (cudaStream_t)h->stream;
    if (h->Fp) {
        if (Fp) {
            if ((e = upload_plane(h, h->Fp, Fp, h->s * h->p.dx * h->p.dx)) != LBM2P_OK)
                return e;
        } else {
            CUDA_TRY(h, cudaMemsetAsync(h->Fp, 0, (size_t)h->plane * sizeof(float), st));
        }
    }
    if (h->Fs) {
        if (Fs) {
            if ((e = upload_plane(h, h->Fs, Fs, h->p.dt)) != LBM2P_OK)
                return e;
        } else {
            CUDA_TRY(h, cudaMemsetAsync(h->Fs, 0, (size_t)h->plane * sizeof(float), st));
        }
    }
    return LBM2P_OK;
}

lbm2p_status lbm2p_set_dirichlet(lbm2p *h, int side, const double *P_b, const double *S_b)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (side < 0 || side > 3 || h->p.bc[side] != LBM2P_BC_DIRICHLET)
        return fail(h, LBM2P_EINVAL, "side %d is not a Dirichlet side", side);
    lbm2p_status e;
    if ((e = upload_trace(h, h->Pb[side], P_b, trace_len(h, side))) != LBM2P_OK)
        return e;
    return upload_trace(h, h->Sb[side], S_b, trace_len(h, side));
}

lbm2p_status lbm2p_step(lbm2p *h, int nsteps, const int *replay, lbm2p_step_stats *stats)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (nsteps < 0)
        return fail(h, LBM2P_EINVAL, "nsteps must be >= 0");
    if (replay)
        for (int s = 0; s < nsteps; ++s)
            if (replay[s] < 0)
                return fail(h, LBM2P_EINVAL, "replay counts must be >= 0");
    lbm2p_status worst = LBM2P_OK;
    for (int s = 0; s < nsteps; ++s) {
        lbm2p_status st = one_step(h, replay ? replay[s] : -1, stats ? stats + s : nullptr);
        if (st != LBM2P_OK && st != LBM2P_ENOTCONVERGED)
            return st;
        if (st != LBM2P_OK)
            worst = st;
    }
    return worst;
}

lbm2p_status lbm2p_pressure_sweeps(lbm2p *h, int nsweeps, double *residual)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (nsweeps < 0)
        return fail(h, LBM2P_EINVAL, "nsweeps must be >= 0");
    double r = std::nan("");
    int pout = h->cur_f;
    lbm2p_status st = pressure_solve(h, nsweeps, false, nullptr, &r, nullptr, &pout);
    h->cur_f = pout;
    if (residual)
        *residual = r;
    return st;
}

static lbm2p_status run_fields(lbm2p *h, float *P, float *S, float *ux, float *uy, int on_device,
                               int mean_free_P)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    cudaStream_t st = (cudaStream_t)h->stream;
    const long long n = h->nnodes;
    float *outs[4] = {P, S, ux, uy};
    float *dst[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int c = 0; c < 4; ++c)
        if (outs[c])
            dst[c] = on_device ? outs[c] : h->stage + (size_t)c * n;
    FieldsArgs a{};
    for (int i = 0; i < 8; ++i)
        a.fin[i] = h->fbuf[h->cur_f][i];
    a.R = R_of(h, false);
    a.inv_tau = itau_of(h, false);
    a.K = h->K;
    a.S = h->S;
    for (int s = 0; s < 4; ++s)
        a.Pb[s] = h->Pb[s];
    a.P_out = dst[0];
    a.S_out = dst[1];
    a.ux_out = dst[2];
    a.uy_out = dst[3];
    a.g = h->geom;
    a.m = h->model;
    lbm2p_launch::fields(a, h->grid, h->stream);
    LAUNCHED(h, "fields");
    if (P && mean_free_P) {
        lbm2p_launch::sum_compact(dst[0], n, h->partials, h->grid, h->stream);
        LAUNCHED(h, "sum");
        lbm2p_launch::finalize_mean(h->partials, h->grid, n, h->mean, h->stream);
        LAUNCHED(h, "mean");
        lbm2p_launch::subtract_mean(dst[0], n, h->mean, h->grid, h->stream);
        LAUNCHED(h, "subtract mean");
    }
    if (!on_device)
        for (int c = 0; c < 4; ++c)
            if (outs[c])
                CUDA_TRY(h, cudaMemcpyAsync(outs[c], dst[c], (size_t)n * sizeof(float),
                                            cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return LBM2P_OK;
}

lbm2p_status lbm2p_velocity(lbm2p *h, float *ux, float *uy, int on_device)
{
    return run_fields(h, nullptr, nullptr, ux, uy, on_device, 0);
}

lbm2p_status lbm2p_fields(lbm2p *h, float *P, float *S, int mean_free_P, int on_device)
{
    return run_fields(h, P, S, nullptr, nullptr, on_device, mean_free_P);
}

size_t lbm2p_state_count(const lbm2p *h)
{
    return h ? (size_t)kStatePlanes * (size_t)h->nnodes : 0;
}

static lbm2p_status state_copy(lbm2p *h, float *buf, size_t count, int on_device, bool out)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (!buf || count != lbm2p_state_count(h))
        return fail(h, LBM2P_EINVAL, "state buffer must hold %zu floats", lbm2p_state_count(h));
    cudaStream_t st = (cudaStream_t)h->stream;
    float *planes[kStatePlanes];
    for (int i = 0; i < 8; ++i)
        planes[i] = h->fbuf[h->cur_f][i];
    for (int i = 0; i < 9; ++i)
        planes[8 + i] = h->gbuf[h->cur_g][i];
    planes[17] = itau_of(h, false);
    planes[18] = h->S;
    planes[19] = R_of(h, false);
    const size_t row = (size_t)h->nx * sizeof(float);
    const size_t dpitch = (size_t)h->pitch * sizeof(float);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                          : (out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    for (int c = 0; c < kStatePlanes; ++c) {
        float *hb = buf + (size_t)c * h->nnodes;
        if (out)
            CUDA_TRY(h, cudaMemcpy2DAsync(hb, row, planes[c], dpitch, row, (size_t)h->ny, kind, st));
        else
            CUDA_TRY(h, cudaMemcpy2DAsync(planes[c], dpitch, hb, row, row, (size_t)h->ny, kind, st));
    }
    if (!out && h->p.warm_start)       // a new state has no history: no extrapolation next step
        CUDA_TRY(h, cudaMemcpyAsync(Pstep_of(h, false), R_of(h, false),
                                    (size_t)h->plane * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return LBM2P_OK;
}

lbm2p_status lbm2p_warm_start(lbm2p *h, const float *P_guess, int on_device)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (!P_guess)
        return fail(h, LBM2P_EINVAL, "P_guess must not be NULL");
    cudaStream_t st = (cudaStream_t)h->stream;
    const size_t row = (size_t)h->nx * sizeof(float);
    CUDA_TRY(h, cudaMemcpy2DAsync(R_of(h, false), (size_t)h->pitch * sizeof(float), P_guess, row, row,
                                  (size_t)h->ny,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    return LBM2P_OK;
}

lbm2p_status lbm2p_get_state(lbm2p *h, float *buf, size_t count, int on_device)
{
    return state_copy(h, buf, count, on_device, true);
}

lbm2p_status lbm2p_set_state(lbm2p *h, const float *buf, size_t count, int on_device)
{
    return state_copy(h, const_cast<float *>(buf), count, on_device, false);
}

lbm2p_status lbm2p_set_timing(lbm2p *h, int enable)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    h->timing = enable != 0;
    return LBM2P_OK;
}

lbm2p_status lbm2p_sweep_config(const lbm2p *h, int *fused, int *kind, int *tile_w, int *tile_h)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (fused)
        *fused = h->tb_T > 1 ? h->tb_T : 1;
    if (h->fp16) {                       // the FP16 sweep kernels
        if (kind)
            *kind = h->h16_kind == 1 ? LBM2P_SWEEP_ROWS : LBM2P_SWEEP_SCALAR;
        if (tile_w)
            *tile_w = h->h16_kind == 1 ? h->h16_w : 0;
        if (tile_h)
            *tile_h = h->h16_kind == 1 ? h->h16_H : 0;
        return LBM2P_OK;
    }
    if (kind)
        *kind = h->sweep_kind + 1;        // internal 0, 1, 2 = VEC4, SCALAR, ROWS
    if (tile_w)
        *tile_w = h->tb_T > 1 ? h->tb_W : (h->sweep_kind == 2 ? h->rows_w : 0);
    if (tile_h)
        *tile_h = h->tb_T > 1 ? h->tb_H : (h->sweep_kind == 2 ? h->rows_H : 0);
    return LBM2P_OK;
}

lbm2p_status lbm2p_set_fused_shape(lbm2p *h, int form, int warps, int slots, int rows)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (h->fp16)
        return fail(h, LBM2P_EINVAL, "FP16 storage sweeps one sweep per launch");
    for (int sd = 0; sd < 4; ++sd)
        if (h->p.bc[sd] == LBM2P_BC_PERIODIC)
            return fail(h, LBM2P_EINVAL, "the two-sweep row-walking kernels need walls on every side");
    // rows per block: a size the create-time tuning tries, clamped to ny as it is there (so a
    // height above ny means ny)
    if (rows > h->ny)
        rows = h->ny;
    auto rows_ok = [&](std::initializer_list<int> tried) {
        for (int H : tried)
            if (rows == (H < h->ny ? H : h->ny))
                return true;
        return false;
    };
    long long grid = 0;
    if ((form == LBM2P_FUSED_STAGED_ROWS && !rows_ok({16, 32, 64, 128})) ||
        (form == LBM2P_FUSED_DIRECT && !rows_ok({2, 4, 8, 16, 32})))
        return fail(h, LBM2P_EINVAL, "rows %d: not a block height of this form for ny = %d", rows,
                    h->ny);
    if (form == LBM2P_FUSED_STAGED_ROWS) {
        if (!lbm2p_launch::rows2_shape_ok(warps, slots))
            return fail(h, LBM2P_EINVAL, "no staged-rows shape with %d consumer warps and %d slots",
                        warps, slots);
        CUDA_TRY(h, lbm2p_launch::rows2_prepare(warps, slots));
        if (lbm2p_launch::rows2_blocks_per_sm(warps, slots, h->Fp != nullptr) < 1)
            return fail(h, LBM2P_EINVAL, "the staged-rows shape does not fit on an SM");
        grid = lbm2p_launch::rows2_grid(warps, rows, h->nx, h->ny);
    } else if (form == LBM2P_FUSED_DIRECT) {
        if ((warps != 4 && warps != 8) || slots != 0)
            return fail(h, LBM2P_EINVAL, "the direct-load form takes 4 or 8 warps and 0 slots");
        grid = lbm2p_launch::pair_direct_grid(warps, rows, h->nx, h->ny);
    } else {
        return fail(h, LBM2P_EINVAL, "form %d cannot be pinned (STAGED_ROWS or DIRECT)", form);
    }
    if (grid > h->partials_cap)
        return fail(h, LBM2P_EINVAL, "%lld blocks exceed the %lld residual partials held", grid,
                    h->partials_cap);
    CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)h->stream));
    drop_graphs(h);
    h->tb_T = 2;
    // as at create: the graph loop body runs the fused launches only when check_every is a
    // multiple of 2 T (an even number of launches per body)
    h->tb_T_graph = h->p.check_every % 4 == 0 ? 2 : 0;
    h->tb_kind = form == LBM2P_FUSED_STAGED_ROWS ? 1 : 2;
    h->tb_W = 30 * warps;
    h->tb_slots = form == LBM2P_FUSED_STAGED_ROWS ? slots : 0;
    h->tb_H = rows;
    h->tb_grid = (int)grid;
    return LBM2P_OK;
}

int lbm2p_fused_form_of(const lbm2p *h)
{
    if (!h || h->fp16 || h->tb_T <= 1)
        return LBM2P_FUSED_NONE;
    return h->tb_kind == 2 ? LBM2P_FUSED_DIRECT
                           : (h->tb_kind == 1 ? LBM2P_FUSED_STAGED_ROWS : LBM2P_FUSED_STAGES);
}

const char *lbm2p_autotune_report(const lbm2p *h)
{
    return h ? h->autotune_log.c_str() : "";
}

lbm2p_status lbm2p_counters(const lbm2p *h, long long *launches, long long *sweeps)
{
    if (!h)
        return fail(nullptr, LBM2P_EINVAL, "NULL handle");
    if (launches)
        *launches = h->launches;
    if (sweeps)
        *sweeps = h->sweeps;
    return LBM2P_OK;
}

const char *lbm2p_last_error(const lbm2p *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

void lbm2p_destroy(lbm2p *h)
{
    if (!h)
        return;
    cudaStreamSynchronize((cudaStream_t)h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"
