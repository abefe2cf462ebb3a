// Device-side definitions shared by the solver's kernels and its runtime: the D2Q9
// lattice, the mobility laws, and the argument blocks passed to each kernel by value.
//
// D2Q9 (Eqs. 3-5, 3-5a, 3-6): c_0 = (0,0); c_1..c_4 = (1,0), (0,1), (-1,0), (0,-1);
// c_5..c_8 = (1,1), (-1,1), (-1,-1), (1,-1); weights 4/9, 1/9, 1/36; pressure source
// weights 0, 1/8 (x8); c_s^2 = 1/3 in lattice units.
//
// Storage (structure of arrays, row pitch padded to 32 floats):
//   f: 8 planes, direction p + 1 in plane p, stored as deviations from a reference
//      pressure R(x):  n_i(x) = f_i^+(x) - w_i R(x).  R is fixed during the pressure
//      sub-iteration of a step and moved to the step's pressure afterwards ("rebase"), so
//      the stored values are the small non-equilibrium and increment parts of f and FP32
//      resolves them finely.  Every sweep works on a_i = f_i(x) - w_i R(x) (pulled value
//      relative to the node's own reference) and dP = P - R(x); because f^eq is linear in
//      P, the collision keeps its form: n_i^+ = a_i + (w_i dP - a_i)/tau_f + F~_p/8.
//      f_0 is never stored: it enters neither P (Eq. 3-9a sums i = 1..8), nor grad P
//      (c_0 = 0), nor any other f_i.
//   g: 9 planes, g_0 .. g_8, plain post-collision values.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm2p.h"

namespace lbm2p_dev {

constexpr int kBlock = 256;   // threads per block of every lattice kernel
constexpr int kMaxWells = LBM2P_MAX_WELLS;

enum : int { BC_PERIODIC = 0, BC_NOFLUX = 1, BC_DIRICHLET = 2 };
enum : int { MOB_QUADRATIC = 0, MOB_DECOUPLED = 1, MOB_RATIONAL = 2 };

__host__ __device__ constexpr int cx(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
__host__ __device__ constexpr float wgt(int i)
{
    return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "diagonal opposites");
static_assert(cx(5) == 1 && cy(5) == 1 && cx(7) == -1 && cy(7) == -1, "diagonals");

// Geometry of one lattice.
struct Geom {
    int nx, ny, pitch;   // pitch in floats
    int tiles_x;         // ceil(nx / kBlock)
    int ntiles;          // tiles_x * ny
    int bc[4];           // XMIN, XMAX, YMIN, YMAX
};

// Physical coefficients, already folded into lattice units by the host.
struct Model {
    int mobility;
    float inv_mu_w, inv_mu_n;
    float phi, inv_phi;
    float s3;            // tau_f = 1/2 + s3 * D_p          (3 s)
    float fs_scale;      // F~_s = fs_scale * F_s          (dt)
    float inv_tau_g;     // 1 / tau_g
    float src_g;         // 1 - 1/(2 tau_g)
    float gam_c;         // gamma~ = -gam_c * lambda_w K   (3 dt / dx^2)
    float inv_dx;
    float Gam[9];        // g_i^eq / S (Eq. 3-4, or Eq. 3-4b on D2Q5)
    int qs;              // saturation lattice: 9 or 5 populations
    float wg[9];         // weights of the saturation lattice (D2Q5: 1/3, 1/6)
    int var_ds;          // tau_g per node: 1/2 + ds_a0 + ds_a1 K lambda_w lambda_n / lambda_t
    float ds_a0, ds_a1;  // 3 D_s dt / (beta dx^2), 3 D_c dt / (beta dx^2)
};

// Sparse point wells, rates already divided by dx^2.
struct Wells {
    int n;
    int idx[kMaxWells];      // j * pitch + i
    float fp[kMaxWells];     // pressure source in lattice units (+- s q)
    float qs[kMaxWells];     // dt q / dx^2 (saturation source magnitude)
    int producer[kMaxWells];
};

struct PressureArgs {
    const float *fin[8];     // n_i of the previous sweep
    float *fout[8];
    const float *R;          // reference pressure of this step
    const float *inv_tau;
    const float *Fp;         // dense F~_p plane (lattice units) or nullptr
    float *Pio;              // pressure plane written (WRITE_P) / read (CHECK)
    double *partials;        // CHECK: 4 doubles per block
    const float *shift;      // CHECK: [0] subtracted from P, [1] from dP - dP_prev, before squaring
    const float *Pb[4];      // Dirichlet traces (device FP32) or nullptr
    Geom g;
    Wells w;
};

struct RefreshArgs {        // stream g, S^n, 1/tau_f (and the warm start of the next solve)
    const float *gin[9];
    const float *Rin;        // reference pressure of the last step
    float *Rout;             // that of the coming solve: Rin, or with the warm start
    const float *Pstep_in;   // 2 Rin - Pstep_in (Pstep_out <- Rin); Pstep_in NULL: no warm
    float *Pstep_out;        // start (Rout <- Rin, nothing when Rout is Rin)
    const float *K;
    const float *Fs;         // dense F~_s plane or nullptr
    float *inv_tau;
    const float *Sb[4];
    Geom g;
    Model m;
    Wells w;
};

struct SaturationArgs {     // stream f and g, grad P, collide g
    const float *fin[8];
    const float *R;
    float *Pnew;             // P of the converged pressure state (for the rebase)
    const float *gin[9];
    float *gout[9];
    const float *K;
    const float *inv_tau;
    const float *Fs;
    float *S;                // S^n written here
    const float *Pb[4];
    const float *Sb[4];
    Geom g;
    Model m;
    Wells w;
};

struct InitGArgs {          // Eqs. gini, gneq and the t = 0 collision
    const float *fin[8];
    const float *R;
    float *Pnew;
    float *gout[9];
    const float *K;
    const float *inv_tau;
    const float *Fs;
    const float *S0;         // initial saturation (read at the node and its neighbours)
    float *S;                // out: S(t=0) from the initial g
    const float *Pb[4];
    const float *Sb[4];
    Geom g;
    Model m;
    Wells w;
};

struct FieldsArgs {         // P, S, u into compact [ny][nx] outputs
    const float *fin[8];
    const float *R;
    const float *inv_tau;
    const float *K;
    const float *S;
    const float *Pb[4];
    float *P_out, *S_out, *ux_out, *uy_out;   // any may be nullptr
    Geom g;
    Model m;
};

struct RebaseArgs {         // n_i += w_i (R - Pnew); R = Pnew  (node-local)
    float *n[8];
    float *R;
    const float *Pnew;
    Geom g;
};

struct RebaseMidArgs {      // within a long solve: R += dP of the last sweep (node-local)
    float *n[8];
    float *R;
    const float *Fp;
    Geom g;
    Wells w;
};

// FP16 storage inside a sub-iteration (fp16.cu)
struct HalfConvertArgs {
    const float *n32[8];     // narrow: FP32 deviations read
    float *n32w[8];          // widen: FP32 deviations written (the same planes)
    __half *n16[8];          // FP16 populations, scaled by scale[0]
    float *R;                // narrow reads it
    float *Rw;               // widen writes it (may be R)
    float *Rh;               // narrow writes it, widen reads it
    float *scale;            // [0] s, [1] 1/s, [2] max |n_i| (as float bits, for the next s)
    Geom g;
};

struct HalfSweepArgs {
    const __half *nin[8];
    __half *nout[8];
    const float *Rin;        // node pressures of the previous sweep
    float *Rout;             // Rin + dP
    const float *inv_tau;
    const float *Fp;
    double *partials;
    const float *shift;
    const float *scale;      // [0] s, [1] 1/s
    float *scale_out;        // the same array: check sweeps raise [3] to max |stored value|
    const float *Pb[4];
    Geom g;
    Wells w;
};

struct ResidualOut {        // written by the finalize kernel
    double r;
    double mean_P;
    double sums[4];
};

// Device-side control of the graph-resident sub-iteration loop.
struct LoopCtl {
    int k;          // sweeps run so far in this solve
    int m;          // sweeps per loop body (= check_every)
    int cap;        // max_sub_iters (a multiple of m)
    int every;      // sweeps between mid-solve rebases (a multiple of m)
    double tol;
    double r;       // last residual
};

}  // namespace lbm2p_dev

// Error text for calls made without a handle (read back by lbm2p_last_error(NULL)).
namespace lbm2p_internal {
lbm2p_status set_global_error(lbm2p_status st, const char *fmt, ...);
}

// Launchers implemented in kernels.cu and sweep_rows.cu (all asynchronous on `stream`).
namespace lbm2p_launch {
using namespace lbm2p_dev;
// single-sweep kernels: kind 0 = four nodes per thread (float4), kind 1 = one node per thread
int max_blocks_per_sm_pressure(bool check, int kind);
void pressure_sweep(const PressureArgs &a, bool check, bool write_p, int grid, void *stream,
                    int kind = 0);
void residual_finalize(const double *partials, int nparts, long long nnodes, float *shift,
                       ResidualOut *out, void *stream);
// T pressure sweeps fused in one launch (T = 2 or 4), W threads per block (a multiple of
// 32, at most 128) owning W - 2T columns, H rows per block; grid = tb_grid(...)
size_t tb_smem_bytes(int T, int W);
long long tb_grid(int T, int W, int H, int nx, int ny);
cudaError_t tb_prepare(int T, int W);
int tb_blocks_per_sm(int T, int W);
void pressure_sweeps_fused(const PressureArgs &a, int T, int W, int H, bool check, int grid,
                           void *stream);
// staged-rows single sweep (sweep_rows.cu): strips of `width` columns (128 or 256; one
// consumer warp per 32 columns plus a producer warp), `slots` ring slots (8; or 6 with width
// 256), H rows per block
bool rows_shape_ok(int width, int slots);
int rows_threads(int width);
size_t rows_smem_bytes(int width, int slots, bool has_fp);
long long rows_grid(int width, int H, int nx, int ny);
cudaError_t rows_prepare(int width, int slots);
int rows_blocks_per_sm(int width, int slots, bool has_fp);
void pressure_sweep_rows(const PressureArgs &a, bool check, bool write_p, int width, int slots,
                         int H, int grid, void *stream);
cudaError_t node_pressure_rows(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                               const PressureArgs &a, bool check, bool write_p, int width,
                               int slots, int H, int grid);
// two sweeps per launch on staged rows (sweep_rows.cu), lattices without periodic sides:
// cw consumer warps of 30 owned columns each (4 or 8), ring slots (6/8 with 4 warps, 4/6
// with 8), H output rows per block; grid = rows2_grid(...)
// slots + kRows2Dense: the (4 warps, 6 slots) shape whose plain launch keeps seven blocks per SM
constexpr int kRows2Dense = LBM2P_ROWS2_DENSE;
bool rows2_shape_ok(int cw, int slots);
int rows2_width(int cw);
size_t rows2_smem_bytes(int cw, int slots, bool has_fp);
long long rows2_grid(int cw, int H, int nx, int ny);
cudaError_t rows2_prepare(int cw, int slots);
int rows2_blocks_per_sm(int cw, int slots, bool has_fp);
void pressure_sweeps_rows2(const PressureArgs &a, bool check, int cw, int slots, int H, int grid,
                           void *stream);
cudaError_t node_pressure_rows2(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                                const PressureArgs &a, bool check, int cw, int slots, int H,
                                int grid);
// two sweeps per launch with direct loads (sweep_rows.cu), lattices without periodic sides:
// cw warps of 30 owned columns (4 or 8), H rows per block; grid = pair_direct_grid(...)
long long pair_direct_grid(int cw, int H, int nx, int ny);
// the direct-load two-sweep kernel (4 warps) over several lattices: item t of items[0 ..
// *nitems) = (member m, block b of m's lattice, strips of 120 columns x H[m] rows), argument
// block pa[2 m + parity]; CHECK: residual sums of the item at parts + 4 (pb0[m] + b)
int pair_batch_blocks_per_sm();
cudaError_t node_pair_batch(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            const PressureArgs *pa, const int *H, const int *pb0,
                            const int2 *items, const int *nitems, int parity, bool check,
                            double *parts, int grid);
void pressure_sweeps_pair_direct(const PressureArgs &a, bool check, int cw, int H, int grid,
                                 void *stream);
cudaError_t node_pressure_pair_direct(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                                      const PressureArgs &a, bool check, int cw, int H, int grid);
// FP16 storage (fp16.cu): narrow = max |n| -> scale -> convert; one sweep; widen
int max_blocks_per_sm_pressure_h();
void half_narrow(const HalfConvertArgs &a, int grid, void *stream);
void half_widen(const HalfConvertArgs &a, int grid, void *stream);
void half_rescale(const HalfConvertArgs &a, float factor, int grid, void *stream);
void pressure_sweep_h(const HalfSweepArgs &a, bool check, int grid, void *stream);
// the FP16 staged-rows sweep (fp16.cu): shapes as for rows_* (width 128 or 256, slots 6 or 8)
size_t rows_h_smem_bytes(int width, int slots, bool has_fp);
cudaError_t rows_h_prepare(int width, int slots);
int rows_h_blocks_per_sm(int width, int slots, bool has_fp);
void pressure_sweep_rows_h(const HalfSweepArgs &a, bool check, int width, int slots, int H,
                           int grid, void *stream);
void refresh(const RefreshArgs &a, int grid, void *stream);
void saturation(const SaturationArgs &a, int grid, void *stream);
void init_g(const InitGArgs &a, int grid, void *stream);
void rebase(const RebaseArgs &a, int grid, void *stream);
void tau_from_S(float *inv_tau, const float *S, const float *K, Geom g, Model m, int grid,
                void *stream);
void fields(const FieldsArgs &a, int grid, void *stream);
// graph nodes (explicit construction; parameters are copied into the node)
cudaError_t node_pressure(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                          const PressureArgs &a, bool check, bool write_p, int grid, int kind);
cudaError_t node_pressure_fused(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                                const PressureArgs &a, int T, int W, int H, bool check, int grid);
cudaError_t node_finalize_loop(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                               const double *partials, int nparts, long long nnodes, float *shift,
                               ResidualOut *out, LoopCtl *ctl, cudaGraphConditionalHandle h,
                               cudaGraphConditionalHandle h_rebase);
void rebase_mid(const RebaseMidArgs &a, int grid, void *stream);
cudaError_t node_rebase_mid(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            const RebaseMidArgs &a, int grid);
cudaError_t node_loop_reset(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            LoopCtl *ctl);
// sets the condition of an IF node: 1 when the loop's last residual is a number
cudaError_t node_if_finite(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                           const LoopCtl *ctl, cudaGraphConditionalHandle h);
cudaError_t node_refresh(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                         const RefreshArgs &a, int grid);
cudaError_t node_saturation(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            const SaturationArgs &a, int grid);
cudaError_t node_rebase(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                        const RebaseArgs &a, int grid);
void sum_compact(const float *x, long long n, double *partials, int grid, void *stream);
void finalize_mean(const double *partials, int nparts, long long n, double *mean, void *stream);
void subtract_mean(float *x, long long n, const double *mean, int grid, void *stream);
}  // namespace lbm2p_launch
