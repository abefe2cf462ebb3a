// The solver handle (private to the library's host code).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm2p.h"
#include "lbm2p_device.cuh"

namespace lbm2p_internal {
struct Alloc {
    void *ptr;
    size_t bytes;
};
}  // namespace lbm2p_internal

struct lbm2p {
    lbm2p_params p{};
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;       // floats per plane
    long long nnodes = 0;
    lbm2p_dev::Geom geom{};
    lbm2p_dev::Model model{};
    lbm2p_dev::Wells wells{};
    double s = 0, tau_g = 0, D_ref = 0;
    int grid = 0;              // blocks of every grid-stride lattice launch
    int grid_check = 0;        // blocks of a pressure sweep that accumulates the residual
    int sweep_kind = 0;        // single-sweep kernel: 0 = four nodes per thread, 1 = one
                               // node per thread, 2 = staged rows
    int grid_sweep = 0;        // blocks of a single sweep without the residual (autotuned)
    long long partials_cap = 0;   // residual partials the partials array holds
    int grid_k[2] = {}, grid_check_k[2] = {}, grid_cap_k[2] = {};
    int rows_w = 0, rows_slots = 0, rows_H = 0, rows_grid = 0;   // staged-rows kernel shape
    int tb_T = 0, tb_W = 0, tb_H = 0, tb_grid = 0;   // fused sweeps per launch and tile shape
    int tb_kind = 0;           // fused kernel: 0 = k_pressure_tb (shared-memory stages), 1 =
                               // k_pressure_rows2 (two sweeps on staged rows), 2 =
                               // k_pressure_pair_direct (two sweeps, direct loads); for 1 and
                               // 2 tb_W = 30 x warps
    int tb_slots = 0;          // ring slots of k_pressure_rows2
    int tb_T_graph = 0;        // fused sweeps used inside the graph loop body (0: single sweeps)
    bool fp16 = false;         // storage FP16_DEV: sweeps run on FP16 copies inside a solve
    __half *hbuf[2][8] = {};
    float *Rh[2] = {};
    float *hscale = nullptr;   // [0] s, [1] 1/s, [2] max |n| of the last narrow,
                               // [3] max |stored value| seen by the check sweeps
    float *hscale_host = nullptr;   // pinned copy
    int hcur = 0;
    int grid_h = 0;            // one-node-per-thread FP16 sweep
    int h16_kind = 0;          // FP16 sweep kernel: 0 one node per thread, 1 staged rows
    int h16_w = 0, h16_slots = 0, h16_H = 0, h16_grid = 0;
    int rebase_every = 0;      // a long solve moves R to the current P after every this many
                               // sweeps (a multiple of check_every)
    void *stream = nullptr;
    std::vector<lbm2p_internal::Alloc> allocs;
    // Pressure populations: three buffers.  A step's solve reads the buffer holding the state
    // (cur_f) and ping-pongs between the other two, so the state it started from is intact
    // until the step succeeds (ENONFINITE leaves every input of the step as it was).
    float *fbuf[3][8] = {};
    float *gbuf[2][9] = {};
    float *K = nullptr, *S = nullptr, *Pio = nullptr, *tmp = nullptr;
    // 1/tau_f, the reference pressure R of the pressure populations, and (warm start) the node
    // pressure of the previous step: two buffers each, cur_r the current one.  A step's S
    // refresh writes the other (the "work" buffer), which becomes current when the step ends.
    float *inv_taub[2] = {};
    float *Rb[2] = {};
    float *Pstepb[2] = {};
    float *Fp = nullptr, *Fs = nullptr;
    float *Pb[4] = {}, *Sb[4] = {};
    double *partials = nullptr, *mean = nullptr;
    float *shift = nullptr;
    lbm2p_dev::ResidualOut *res = nullptr;
    lbm2p_dev::ResidualOut *res_host = nullptr;   // pinned
    float *stage = nullptr;            // compact [ny][nx] device staging plane
    int cur_f = 0, cur_g = 0;          // buffers holding the current post-collision state
    int cur_r = 0;                     // current buffer of 1/tau_f, R and the previous P
    long long launches = 0, sweeps = 0;
    bool timing = false;
    cudaEvent_t ev_step0 = nullptr, ev_step1 = nullptr, ev_sw0 = nullptr, ev_sw1 = nullptr;
    // graph-resident sub-iteration (free-running solves when check_every is even and
    // divides max_sub_iters): one graph per (f buffer, R buffer) for a bare solve, and one per
    // (f buffer, g buffer, R buffer) for a whole physical step
    bool graph_ok = false;
    lbm2p_dev::LoopCtl *ctl = nullptr;
    lbm2p_dev::LoopCtl *ctl_host = nullptr;       // pinned
    cudaGraph_t solve_g[3][2] = {};
    cudaGraphExec_t solve_x[3][2] = {};
    cudaGraph_t step_g[3][2][2] = {};
    cudaGraphExec_t step_x[3][2][2] = {};
    std::string autotune_log;          // one line per candidate timed at create
    std::string err;
};


namespace lbm2p_internal {
// the f buffer k places after b in the rotation of three
inline int fnext(int b, int k) { return (b + k) % 3; }
// 1/tau_f, R and the previous step's P: the current buffers, or the work buffers of a step
inline float *itau_of(const lbm2p *h, bool work) { return h->inv_taub[work ? 1 - h->cur_r : h->cur_r]; }
inline float *R_of(const lbm2p *h, bool work) { return h->Rb[work ? 1 - h->cur_r : h->cur_r]; }
inline float *Pstep_of(const lbm2p *h, bool work) { return h->Pstepb[work ? 1 - h->cur_r : h->cur_r]; }
// kernel argument blocks of h (runtime.cu): sweeps from f buffer src into dst, the S refresh
// of g buffer pg (in place: R, P^{n-1} and 1/tau_f overwritten; otherwise written into the
// work buffers), saturation update and rebases of f buffer pf; `work`: use the work buffers
lbm2p_dev::PressureArgs pressure_args(lbm2p *h, int src, int dst, bool work);
lbm2p_dev::RefreshArgs refresh_args(lbm2p *h, int pg, bool in_place);
lbm2p_dev::SaturationArgs saturation_args(lbm2p *h, int pf, int pg, bool work);
lbm2p_dev::RebaseArgs rebase_args(lbm2p *h, int pf, bool work);
lbm2p_dev::RebaseMidArgs rebase_mid_args(lbm2p *h, int pf, bool work);
}  // namespace lbm2p_internal
