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
    float *fbuf[2][8] = {};
    float *gbuf[2][9] = {};
    float *inv_tau = nullptr, *K = nullptr, *S = nullptr, *Pio = nullptr, *tmp = nullptr;
    float *R = nullptr;                // reference pressure of the pressure populations
    float *Pstep = nullptr;            // warm start: the node pressure of the previous step
    float *Fp = nullptr, *Fs = nullptr;
    float *Pb[4] = {}, *Sb[4] = {};
    double *partials = nullptr, *mean = nullptr;
    float *shift = nullptr;
    lbm2p_dev::ResidualOut *res = nullptr;
    lbm2p_dev::ResidualOut *res_host = nullptr;   // pinned
    float *stage = nullptr;            // compact [ny][nx] device staging plane
    int cur_f = 0, cur_g = 0;          // buffer holding the current post-collision state
    long long launches = 0, sweeps = 0;
    bool timing = false;
    cudaEvent_t ev_step0 = nullptr, ev_step1 = nullptr, ev_sw0 = nullptr, ev_sw1 = nullptr;
    // graph-resident sub-iteration (free-running solves when check_every is even and
    // divides max_sub_iters): one graph per f parity for a bare solve, and one per
    // (f parity, g parity) for a whole physical step
    bool graph_ok = false;
    lbm2p_dev::LoopCtl *ctl = nullptr;
    lbm2p_dev::LoopCtl *ctl_host = nullptr;       // pinned
    cudaGraph_t solve_g[2] = {};
    cudaGraphExec_t solve_x[2] = {};
    cudaGraph_t step_g[2][2] = {};
    cudaGraphExec_t step_x[2][2] = {};
    std::string autotune_log;          // one line per candidate timed at create
    std::string err;
};


namespace lbm2p_internal {
// kernel argument blocks of h for f source parity src / g parity pg (runtime.cu)
lbm2p_dev::PressureArgs pressure_args(lbm2p *h, int src);
lbm2p_dev::RefreshArgs refresh_args(lbm2p *h, int pg);
lbm2p_dev::SaturationArgs saturation_args(lbm2p *h, int pf, int pg);
lbm2p_dev::RebaseArgs rebase_args(lbm2p *h, int pf);
lbm2p_dev::RebaseMidArgs rebase_mid_args(lbm2p *h, int pf);
}  // namespace lbm2p_internal
