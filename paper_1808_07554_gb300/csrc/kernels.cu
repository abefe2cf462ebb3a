// CUDA kernels of the two-phase Darcy LB solver (sm_103a).
//
// Every lattice kernel is a grid-stride loop over row tiles of kBlock nodes (one node per
// thread, consecutive threads on consecutive x): the grid is sized to the resident-block
// capacity of the GPU, so each block sweeps many tiles and the FP64 residual partials stay
// few.  Pull scheme: a node gathers f_i^+(x - c_i) from the previous sweep's buffer and
// writes its own post-collision values into the other buffer (ping-pong), so one launch
// is one fused stream + collide of Eq. 3-1 (or Eq. 3-2).  Wall rules of Sec. 4 are folded
// into the gather: interior nodes take a branch-free path; only nodes on the lattice edge
// evaluate the periodic / bounce-back / anti-bounce-back substitution.  The pressure
// populations are stored as deviations from the step's reference pressure (see
// lbm2p_device.cuh), and every pressure kernel works on those deviations.
#include <cuda_runtime.h>

#include <cmath>

#include "lbm2p_device.cuh"
#include "lbm2p_node.cuh"

namespace lbm2p_dev {

// --------------------------------------------------------------------------------------
// a2/a3: fused pressure sweep (Eq. 3-1), four consecutive nodes per thread (one float4 per
// plane row), a row tile of 4 * kBlock nodes per block iteration.  Directions with c_x = 0
// read their float4 directly; c_x = +1 needs the element left of the float4 (from lane - 1
// by a shuffle, or a scalar load in lane 0), c_x = -1 the element right of it (lane + 1, or
// lane 31's load).  The reference pressure R is gathered the same way.  Threads whose nodes
// touch the lattice edge, whole edge rows and the ragged tail use the scalar gather with the
// wall rules.  CHECK adds the residual partials (dP - dP_prev and P - shift, FP32 per warp,
// FP64 per block); WRITE_P stores dP for the next check.
// --------------------------------------------------------------------------------------
__device__ __forceinline__ float4 ld4(const float *p, int o)
{
    return __ldg(reinterpret_cast<const float4 *>(p + o));
}

__device__ __forceinline__ void st4(float *p, int o, float4 v)
{
    *reinterpret_cast<float4 *>(p + o) = v;
}

// (left neighbour of v.x, v.x, v.y, v.z): the row shifted right by one node
__device__ __forceinline__ float4 shift_in_left(float4 v, const float *row, int o, int lane,
                                                bool has_left)
{
    float l = __shfl_up_sync(0xffffffffu, v.w, 1);
    if (lane == 0)
        l = has_left ? __ldg(row + o - 1) : 0.0f;
    return make_float4(l, v.x, v.y, v.z);
}

// (v.y, v.z, v.w, right neighbour of v.w): the row shifted left by one node
__device__ __forceinline__ float4 shift_in_right(float4 v, const float *row, int o, int lane,
                                                 bool has_right)
{
    float r = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (lane == 31)
        r = has_right ? __ldg(row + o + 4) : 0.0f;
    return make_float4(v.y, v.z, v.w, r);
}

// (left neighbour of v.x, v.x, v.y, v.z): the row shifted right by one node; lane 0 takes
// the element left of the warp from `edge`
__device__ __forceinline__ float4 shl(float4 v, float edge, int lane)
{
    float l = __shfl_up_sync(0xffffffffu, v.w, 1);
    if (lane == 0)
        l = edge;
    return make_float4(l, v.x, v.y, v.z);
}

// (v.y, v.z, v.w, right neighbour of v.w); lane 31 takes the element right of the warp
__device__ __forceinline__ float4 shr(float4 v, float edge, int lane)
{
    float r = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (lane == 31)
        r = edge;
    return make_float4(v.y, v.z, v.w, r);
}

// n + w (r - r0), elementwise
__device__ __forceinline__ float4 dev4(float4 n, float w, float4 r, float4 r0)
{
    return make_float4(dev1(n.x, w, r.x, r0.x), dev1(n.y, w, r.y, r0.y), dev1(n.z, w, r.z, r0.z),
                       dev1(n.w, w, r.w, r0.w));
}

#ifndef LBM2P_SWEEP_MINB
#define LBM2P_SWEEP_MINB 4
#endif
template <bool CHECK, bool WRITE_P>
__global__ void __launch_bounds__(kBlock, LBM2P_SWEEP_MINB) k_pressure(const __grid_constant__ PressureArgs a)
{
    const Geom &g = a.g;
    const int lane = threadIdx.x & 31;
    const int p = g.pitch;
    ResAcc racc;                                      // residual sums of this thread
    const float shift = CHECK ? a.shift[0] : 0.0f;    // constant subtracted from P
    const float dshift = CHECK ? a.shift[1] : 0.0f;   // constant subtracted from dP - dP_prev
    const int tiles_x = (g.nx + 4 * kBlock - 1) / (4 * kBlock);
    const int ntiles = tiles_x * g.ny;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = t / tiles_x;
        const int x0 = ((t - y * tiles_x) * kBlock + threadIdx.x) * 4;
        const int o = y * p + x0;
        const bool row_inner = y > 0 && y < g.ny - 1;     // uniform over the block
        bool fast = false;
        float4 f[8], r0, it, F;
        if (row_inner) {
            // every lane takes part in the shuffles; lanes past the padded row load nothing.
            // All global loads of the tile are issued before any of them is used.
            const bool in_row = x0 < p;
            const bool hl = x0 >= 1 && in_row, hr = x0 + 4 < g.nx;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float *R = a.R;
            float4 v[11];
            if (in_row) {
                v[0] = ld4(a.fin[0], o);          // c = ( 1, 0): row y, shifted right
                v[1] = ld4(a.fin[1], o - p);      // c = ( 0, 1): row y - 1
                v[2] = ld4(a.fin[2], o);          // c = (-1, 0): row y, shifted left
                v[3] = ld4(a.fin[3], o + p);      // c = ( 0,-1): row y + 1
                v[4] = ld4(a.fin[4], o - p);      // c = ( 1, 1)
                v[5] = ld4(a.fin[5], o - p);      // c = (-1, 1)
                v[6] = ld4(a.fin[6], o + p);      // c = (-1,-1)
                v[7] = ld4(a.fin[7], o + p);      // c = ( 1,-1)
                v[8] = ld4(R, o - p);
                v[9] = ld4(R, o);
                v[10] = ld4(R, o + p);
                it = ld4(a.inv_tau, o);
                F = a.Fp ? ld4(a.Fp, o) : z;
            } else {
#pragma unroll
                for (int i = 0; i < 11; ++i)
                    v[i] = z;
                it = z;
                F = z;
            }
            // the elements just left / right of this warp's 128 nodes (lanes 0 and 31)
            float el[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, er[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (lane == 0 && hl) {
                el[0] = __ldg(a.fin[0] + o - 1);
                el[1] = __ldg(a.fin[4] + o - p - 1);
                el[2] = __ldg(a.fin[7] + o + p - 1);
                el[3] = __ldg(R + o - p - 1);
                el[4] = __ldg(R + o - 1);
                el[5] = __ldg(R + o + p - 1);
            }
            if (lane == 31 && hr) {
                er[0] = __ldg(a.fin[2] + o + 4);
                er[1] = __ldg(a.fin[5] + o - p + 4);
                er[2] = __ldg(a.fin[6] + o + p + 4);
                er[3] = __ldg(R + o - p + 4);
                er[4] = __ldg(R + o + 4);
                er[5] = __ldg(R + o + p + 4);
            }
            r0 = v[9];
            const float4 rl = shl(v[9], el[4], lane), rr = shr(v[9], er[4], lane);
            const float4 rml = shl(v[8], el[3], lane), rmr = shr(v[8], er[3], lane);
            const float4 rpl = shl(v[10], el[5], lane), rpr = shr(v[10], er[5], lane);
            // a_i = n_i(x - c_i) + w_i (R(x - c_i) - R(x))
            f[0] = dev4(shl(v[0], el[0], lane), wgt(1), rl, r0);
            f[1] = dev4(v[1], wgt(2), v[8], r0);
            f[2] = dev4(shr(v[2], er[0], lane), wgt(3), rr, r0);
            f[3] = dev4(v[3], wgt(4), v[10], r0);
            f[4] = dev4(shl(v[4], el[1], lane), wgt(5), rml, r0);
            f[5] = dev4(shr(v[5], er[1], lane), wgt(6), rmr, r0);
            f[6] = dev4(shr(v[6], er[2], lane), wgt(7), rpr, r0);
            f[7] = dev4(shl(v[7], el[2], lane), wgt(8), rpl, r0);
            fast = hl && x0 + 4 <= g.nx - 1;
        }
        if (fast) {
            for (int k = 0; k < a.w.n; ++k) {
                const int d = a.w.idx[k] - o;
                if (d >= 0 && d < 4) {
                    if (d == 0) F.x += a.w.fp[k];
                    else if (d == 1) F.y += a.w.fp[k];
                    else if (d == 2) F.z += a.w.fp[k];
                    else F.w += a.w.fp[k];
                }
            }
            float dPv[4];
            float4 out[8];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float fc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    fc[i] = (&f[i].x)[c];
                const float dP = pressure_of(fc);
                const float itc = (&it.x)[c];
                const float Fq = 0.125f * (&F.x)[c];   // w_bar_i = 1/8 (Eq. 3-5a)
                // Eq. 2-1b relative to R: n_i^+ = a_i + (w_i dP - a_i)/tau_f + w_bar_i F~_p
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    (&out[i].x)[c] = collide1(fc[i], wgt(i + 1), dP, itc, Fq);
                dPv[c] = dP;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                st4(a.fout[i], o, out[i]);
            if (CHECK) {
                const float4 Pp = ld4(a.Pio, o);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float d = (dPv[c] - (&Pp.x)[c]) - dshift, q = ((&r0.x)[c] - shift) + dPv[c];
                    racc.add(d, q);
                }
            }
            if (WRITE_P)
                st4(a.Pio, o, make_float4(dPv[0], dPv[1], dPv[2], dPv[3]));
        } else {
            // edge rows, edge columns and the ragged tail: scalar nodes with the wall rules
            for (int c = 0; c < 4; ++c) {
                const int x = x0 + c;
                if (x >= g.nx)
                    break;
                const int oc = o + c;
                float fc[8];
                gather_a(a.fin, a.R, g, a.Pb, x, y, oc, fc);
                const float dP = pressure_of(fc);
                const float itc = a.inv_tau[oc];
                float F = a.Fp ? a.Fp[oc] : 0.0f;
                for (int k = 0; k < a.w.n; ++k)
                    if (oc == a.w.idx[k])
                        F += a.w.fp[k];
                const float Fq = 0.125f * F;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    a.fout[i][oc] = collide1(fc[i], wgt(i + 1), dP, itc, Fq);
                if (CHECK) {
                    const float d = (dP - a.Pio[oc]) - dshift, q = (a.R[oc] - shift) + dP;
                    racc.add(d, q);
                }
                if (WRITE_P)
                    a.Pio[oc] = dP;
            }
        }
    }
    if (CHECK) {
        __shared__ double red[kBlock / 32][4];
        const int warp = threadIdx.x >> 5;
        double v[4];
        racc.warp_totals(v);
        if (lane == 0) {
            red[warp][0] = v[0];
            red[warp][1] = v[1];
            red[warp][2] = v[2];
            red[warp][3] = v[3];
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kBlock / 32; ++w)
                s += red[w][threadIdx.x];
            a.partials[4 * blockIdx.x + threadIdx.x] = s;
        }
    }
}

// --------------------------------------------------------------------------------------
// a2/a3 fused in time: T pressure sweeps per launch.
//
// Block b owns a strip of W = blockDim.x columns and H rows.  It marches down its rows;
// at iteration j it loads input row j+1 (stage 0: the populations of the previous launch)
// into shared memory and computes stage s (the s-th sweep) at row j - s + 1, s = 1..T,
// each stage from the three rows of the stage before it.  Stage s is computed on the
// columns [x0 - (T - s), x0 + W + (T - s)): the halo a stage needs shrinks by one node per
// stage, so stage T covers exactly the owned strip.  Shared memory holds, per stage
// s < T, a ring of its last three rows (8 planes each), the reference pressure R of the
// last T + 2 input rows, and (CHECK) the stage T-1 pressure increments.  Periodic sides
// need no special case: halo loads wrap, so the shared rows hold the periodic images.
// Nodes beyond a wall are skipped, and nodes on a wall apply the wall rules of Sec. 4 to
// their own stage values.  Every node of every stage is computed with the same arithmetic
// as one sweep of k_pressure, so T fused sweeps equal T single sweeps bit for bit; the
// cost is the recomputation of the halo (about 2 (T - 1) / W of the columns and
// 2 (T - 1) / H of the rows) against one read and one write of the populations per T
// sweeps.  CHECK: the residual partials of the last stage against stage T - 1.
// --------------------------------------------------------------------------------------
struct TBLayout {
    int Wt, T;                                     // threads per block, fused sweeps
    // stage s is computed on Wt - 2 s columns: the input row spans all threads and the last
    // stage the Wt - 2 T columns the block owns, so every stage is one pass of the block
    __device__ __forceinline__ int width(int s) const { return Wt - 2 * s; }
    // float offset of stage s's ring (s = 0 .. T-1): 3 rows x 8 planes x width(s)
    __device__ __forceinline__ int ring(int s) const
    {
        int off = 0;
        for (int q = 0; q < s; ++q)
            off += 24 * width(q);
        return off;
    }
    // per-row fields of the last T + 2 input rows (width(0) each): R, 1/tau_f, F~_p
    __device__ __forceinline__ int rring() const { return ring(T); }
    __device__ __forceinline__ int tring() const { return rring() + (T + 2) * width(0); }
    __device__ __forceinline__ int fring() const { return tring() + (T + 2) * width(0); }
    __device__ __forceinline__ int dpring() const { return fring() + (T + 2) * width(0); }
};

__device__ __forceinline__ int wrap_coord(int v, int n) { return ((v % n) + n) % n; }

// one input row's values for the column a thread stages
struct TBRow {
    float v[11];
};

template <int T, bool CHECK>
__global__ void __launch_bounds__(128) k_pressure_tb(const __grid_constant__ PressureArgs a, int H)
{
    extern __shared__ float sm[];
    const Geom &g = a.g;
    const int Wt = blockDim.x;
    const int W = Wt - 2 * T;                      // columns owned by the block
    const TBLayout L{Wt, T};
    const int strips = (g.nx + W - 1) / W;
    const int x0 = (blockIdx.x % strips) * W;
    const int y0 = (blockIdx.x / strips) * H;
    const bool perx = g.bc[0] == BC_PERIODIC, pery = g.bc[2] == BC_PERIODIC;
    const int p = g.pitch;
    const int tid = threadIdx.x;
    const int ylo = y0 - T;                        // local row 0
    const int w0 = L.width(0);
    const float shift = CHECK ? a.shift[0] : 0.0f;
    const float dshift = CHECK ? a.shift[1] : 0.0f;
    ResAcc racc;                                   // residual sums of this thread

    // global loads of input row r (8 planes, R, 1/tau_f, F~_p) at this thread's column
    auto fetch = [&](int r, TBRow &row) {
        const bool vy = pery || (r >= 0 && r < g.ny);
        const int rw = pery ? wrap_coord(r, g.ny) : r;
        const int xl = x0 - T + tid;
        const bool vx = perx || (xl >= 0 && xl < g.nx);
        if (vx && vy) {
            const int o = rw * p + (perx ? wrap_coord(xl, g.nx) : xl);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                row.v[i] = __ldg(a.fin[i] + o);
            row.v[8] = __ldg(a.R + o);
            row.v[9] = __ldg(a.inv_tau + o);
            float F = a.Fp ? __ldg(a.Fp + o) : 0.0f;
            for (int k = 0; k < a.w.n; ++k)
                if (o == a.w.idx[k])
                    F += a.w.fp[k];
            row.v[10] = 0.125f * F;                // w_bar_i F~_p, w_bar_i = 1/8 (Eq. 3-5a)
        } else {
#pragma unroll
            for (int i = 0; i < 11; ++i)
                row.v[i] = 0.0f;
        }
    };
    // registers of input row r into the shared rings
    auto stage_in = [&](int r, const TBRow &row) {
        const int rl = r - ylo;
        float *ring0 = sm + L.ring(0) + (rl % 3) * 8 * w0;
        const int fs = (rl % (T + 2)) * w0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            ring0[i * w0 + tid] = row.v[i];
        sm[L.rring() + fs + tid] = row.v[8];
        sm[L.tring() + fs + tid] = row.v[9];
        sm[L.fring() + fs + tid] = row.v[10];
    };

    TBRow nxt;
    fetch(ylo, nxt);
    stage_in(ylo, nxt);
    fetch(ylo + 1, nxt);
    stage_in(ylo + 1, nxt);
    const int j0 = y0 - T + 1, j1 = y0 + H + T - 2;
    fetch(j0 + 1, nxt);
    for (int j = j0; j <= j1; ++j) {
        stage_in(j + 1, nxt);                  // row j + 1 was fetched one iteration ahead
        __syncthreads();
        if (j + 1 <= j1)
            fetch(j + 2, nxt);                 // in flight while this iteration computes
#pragma unroll
        for (int s = 1; s <= T; ++s) {
            const int r = j - s + 1;
            const int halo = T - s;
            const bool in_range = r >= y0 - halo && r < y0 + H + halo;
            const bool vy = pery || (r >= 0 && r < g.ny);
            if (in_range && vy) {
                const int rw = pery ? wrap_coord(r, g.ny) : r;
                const int rl = r - ylo;
                const float *src = sm + L.ring(s - 1);
                const int ws = L.width(s - 1);
                const int fs_m = ((rl - 1 + (T + 2)) % (T + 2)) * w0, fs_0 = (rl % (T + 2)) * w0,
                          fs_p = ((rl + 1) % (T + 2)) * w0;
                const float *srow_m = src + ((rl - 1 + 3) % 3) * 8 * ws;   // row r - 1
                const float *srow_0 = src + (rl % 3) * 8 * ws;             // row r
                const float *srow_p = src + ((rl + 1) % 3) * 8 * ws;       // row r + 1
                const float *Rm = sm + L.rring() + fs_m, *R0 = sm + L.rring() + fs_0,
                            *Rp = sm + L.rring() + fs_p;
                const float *IT = sm + L.tring() + fs_0, *FQ = sm + L.fring() + fs_0;
                const int c = tid;
                const int xl = x0 - halo + c;
                if (c < L.width(s) && (perx || (xl >= 0 && xl < g.nx))) {
                    const int xw = perx ? wrap_coord(xl, g.nx) : xl;
                    const int cs = c + 1;              // this node in stage s-1 columns
                    const int c0 = c + s;              // this node in input-row columns
                    const float r0 = R0[c0];
                    float f[8];
                    const bool wall = (!perx && (xw == 0 || xw == g.nx - 1)) ||
                                      (!pery && (rw == 0 || rw == g.ny - 1));
                    if (!wall) {
                        // a_i = n_i(x - c_i) + w_i (R(x - c_i) - R(x)), all from shared rows
                        f[0] = dev1(srow_0[0 * ws + cs - 1], wgt(1), R0[c0 - 1], r0);
                        f[1] = dev1(srow_m[1 * ws + cs], wgt(2), Rm[c0], r0);
                        f[2] = dev1(srow_0[2 * ws + cs + 1], wgt(3), R0[c0 + 1], r0);
                        f[3] = dev1(srow_p[3 * ws + cs], wgt(4), Rp[c0], r0);
                        f[4] = dev1(srow_m[4 * ws + cs - 1], wgt(5), Rm[c0 - 1], r0);
                        f[5] = dev1(srow_m[5 * ws + cs + 1], wgt(6), Rm[c0 + 1], r0);
                        f[6] = dev1(srow_p[6 * ws + cs + 1], wgt(7), Rp[c0 + 1], r0);
                        f[7] = dev1(srow_p[7 * ws + cs - 1], wgt(8), Rp[c0 - 1], r0);
                    } else {
#pragma unroll
                        for (int i = 1; i <= 8; ++i) {
                            const int ex = cx(i), ey = cy(i);
                            int side = -1;
                            if (!perx && (xw - ex < 0 || xw - ex >= g.nx))
                                side = xw - ex < 0 ? 0 : 1;
                            else if (!pery && (rw - ey < 0 || rw - ey >= g.ny))
                                side = rw - ey < 0 ? 2 : 3;
                            if (side < 0) {
                                const float *row = ey == 1 ? srow_m : (ey == -1 ? srow_p : srow_0);
                                const float *Rrow = ey == 1 ? Rm : (ey == -1 ? Rp : R0);
                                f[i - 1] = dev1(row[(i - 1) * ws + cs - ex], wgt(i), Rrow[c0 - ex], r0);
                            } else {
                                const float b = srow_0[(opp(i) - 1) * ws + cs];
                                if (g.bc[side] == BC_NOFLUX) {
                                    f[i - 1] = b;
                                } else {
                                    const int k = side < 2 ? 2 * rw + 1 - ey : 2 * xw + 1 - ex;
                                    f[i - 1] = -b + 2.0f * wgt(i) * (a.Pb[side][k] - r0);
                                }
                            }
                        }
                    }
                    const float dP = pressure_of(f);
                    const float it = IT[c0];
                    const float Fq = FQ[c0];
                    if (s < T) {
                        float *dst = sm + L.ring(s) + (rl % 3) * 8 * L.width(s);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            dst[i * L.width(s) + c] = collide1(f[i], wgt(i + 1), dP, it, Fq);
                        if (CHECK && s == T - 1)
                            sm[L.dpring() + (rl % 3) * L.width(T - 1) + c] = dP;
                    } else if (xl >= x0 && xl < x0 + W && xl < g.nx && r >= y0 && r < y0 + H &&
                               r < g.ny && r >= 0) {
                        const int o = rw * p + xw;
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            a.fout[i][o] = collide1(f[i], wgt(i + 1), dP, it, Fq);
                        if (CHECK) {
                            const float d = (dP - sm[L.dpring() + (rl % 3) * L.width(T - 1) + c + 1]) - dshift;
                            const float q = (r0 - shift) + dP;
                            racc.add(d, q);
                        }
                    }
                }
            }
            if (s < T)
                __syncthreads();
        }
        __syncthreads();
    }
    if (CHECK) {
        const int lane = tid & 31, warp = tid >> 5;
        double v[4];
        racc.warp_totals(v);
        __shared__ double red[4][4];
        if (lane == 0) {
            red[warp][0] = v[0];
            red[warp][1] = v[1];
            red[warp][2] = v[2];
            red[warp][3] = v[3];
        }
        __syncthreads();
        if (tid < 4) {
            double acc = 0.0;
            for (int w = 0; w < Wt / 32; ++w)
                acc += red[w][tid];
            a.partials[4 * blockIdx.x + tid] = acc;
        }
    }
}

// One node per thread (row tiles of kBlock nodes): the same sweep with scalar loads and a
// small register footprint (more resident warps); faster where the sweep is latency-bound.
template <bool CHECK, bool WRITE_P>
__global__ void __launch_bounds__(kBlock) k_pressure_scalar(const __grid_constant__ PressureArgs a)
{
    const Geom &g = a.g;
    const int lane = threadIdx.x & 31;
    // residual sums: per thread over its nodes, then per warp and per block once, after the
    // sweep
    ResAcc racc;
    const float shift = CHECK ? a.shift[0] : 0.0f;
    const float dshift = CHECK ? a.shift[1] : 0.0f;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        float d = 0.0f, q = 0.0f;
        if (x < g.nx) {
            sweep_node<CHECK, WRITE_P>(a, x, y, y * g.pitch + x, shift, dshift, d, q);
            if (CHECK)
                racc.add(d, q);
        }
    }
    if (CHECK) {
        __shared__ double red[kBlock / 32][4];
        const int warp = threadIdx.x >> 5;
        double v[4];
        racc.warp_totals(v);
        if (lane == 0) {
            red[warp][0] = v[0];
            red[warp][1] = v[1];
            red[warp][2] = v[2];
            red[warp][3] = v[3];
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int w = 0; w < kBlock / 32; ++w)
                s += red[w][threadIdx.x];
            a.partials[4 * blockIdx.x + threadIdx.x] = s;
        }
    }
}

// r = ||dP - mean dP|| / ||P - mean P|| from the block partials (FP64, fixed order).
// Called by all 256 threads of one block; returns r in thread 0.
__device__ double finalize_residual(const double *__restrict__ partials, int nparts,
                                    long long nnodes, float *shift, ResidualOut *out)
{
    __shared__ double red[256][4];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += 256)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            s[c] += partials[4 * i + c];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        red[threadIdx.x][c] = s[c];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                red[threadIdx.x][c] += red[threadIdx.x + h][c];
        __syncthreads();
    }
    double r = 0.0;
    if (threadIdx.x == 0) {
        const double N = (double)nnodes;
        const double sd = red[0][0], sdd = red[0][1], sp = red[0][2], spp = red[0][3];
        const double c = (double)shift[0], cd = (double)shift[1];
        if (!isfinite(sd) || !isfinite(sdd) || !isfinite(sp) || !isfinite(spp)) {
            r = nan("");
        } else {
            // sums of (dP - dP_prev - cd) and (P - c): variances are shift invariant
            double num = sdd - sd * sd / N;
            double den = spp - sp * sp / N;
            num = num > 0.0 ? num : 0.0;
            den = den > 0.0 ? den : 0.0;
            r = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
            shift[0] = (float)(c + sp / N);
            shift[1] = (float)(cd + sd / N);
        }
        out->r = r;
        out->mean_P = c + sp / N;
        out->sums[0] = sd;
        out->sums[1] = sdd;
        out->sums[2] = sp;
        out->sums[3] = spp;
    }
    return r;
}

__global__ void __launch_bounds__(256) k_residual_finalize(const double *__restrict__ partials,
                                                           int nparts, long long nnodes,
                                                           float *shift, ResidualOut *out)
{
    finalize_residual(partials, nparts, nnodes, shift, out);
}

// Finalize inside the graph-resident loop: count the body's sweeps and keep looping while
// r > tol, r is a number, and the cap is not reached.
__global__ void __launch_bounds__(256) k_residual_finalize_loop(
    const double *__restrict__ partials, int nparts, long long nnodes, float *shift,
    ResidualOut *out, LoopCtl *ctl, cudaGraphConditionalHandle handle,
    cudaGraphConditionalHandle h_rebase)
{
    const double r = finalize_residual(partials, nparts, nnodes, shift, out);
    if (threadIdx.x == 0) {
        const int k = ctl->k + ctl->m;
        ctl->k = k;
        ctl->r = r;
        const bool more = !(r <= ctl->tol) && !isnan(r) && k < ctl->cap;
        cudaGraphSetConditional(handle, more ? 1u : 0u);
        cudaGraphSetConditional(h_rebase, more && ctl->every > 0 && k % ctl->every == 0 ? 1u : 0u);
    }
}

__global__ void k_loop_reset(LoopCtl *ctl)
{
    ctl->k = 0;
    ctl->r = nan("");
}

// After the loop: the step goes on (saturation update, rebase) only when the last residual is
// a number; otherwise the step's inputs stay as they were and the host reports ENONFINITE.
__global__ void k_if_finite(const LoopCtl *ctl, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, isnan(ctl->r) ? 0u : 1u);
}

// --------------------------------------------------------------------------------------
// a1: stream g, S^n (Eq. 3-9b), 1/tau_f (Eq. 3-11a with D_p = K lambda_t(S))
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_refresh(const __grid_constant__ RefreshArgs a)
{
    const Geom &g = a.g;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx)
            refresh_node(a, x, y, y * g.pitch + x);
    }
}

// --------------------------------------------------------------------------------------
// a4 + a5: local grad P (Eq. 3-10a) and the fused saturation stream + collide (Eq. 3-2)
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_saturation(const __grid_constant__ SaturationArgs a)
{
    const Geom &g = a.g;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx)
            saturation_node(a, x, y, y * g.pitch + x);
    }
}

// --------------------------------------------------------------------------------------
// a6: initial g (Eqs. gini, gneq) followed by the t = 0 collision
// --------------------------------------------------------------------------------------
__device__ __forceinline__ float s_at(const float *S, const Geom &g, int x, int y)
{
    return S[y * g.pitch + x];
}

// central difference of S0 along one axis in lattice units; mirror at no-flux walls,
// wrap if periodic, second-order one-sided at Dirichlet walls
__device__ float fd_axis(const float *S, const Geom &g, int x, int y, int axis)
{
    const int n = axis == 0 ? g.nx : g.ny;
    const int c = axis == 0 ? x : y;
    const int lo_side = axis == 0 ? 0 : 2, hi_side = lo_side + 1;
    auto at = [&](int cc) { return axis == 0 ? s_at(S, g, cc, y) : s_at(S, g, x, cc); };
    if (c == 0 && g.bc[lo_side] == BC_DIRICHLET)
        return (-3.0f * at(0) + 4.0f * at(1) - at(2)) * 0.5f;
    if (c == n - 1 && g.bc[hi_side] == BC_DIRICHLET)
        return (3.0f * at(n - 1) - 4.0f * at(n - 2) + at(n - 3)) * 0.5f;
    const float lo = c - 1 >= 0 ? at(c - 1) : (g.bc[lo_side] == BC_PERIODIC ? at(n - 1) : at(c));
    const float hi = c + 1 < n ? at(c + 1) : (g.bc[hi_side] == BC_PERIODIC ? at(0) : at(c));
    return (hi - lo) * 0.5f;
}

__global__ void __launch_bounds__(kBlock) k_init_g(const __grid_constant__ InitGArgs a)
{
    const Geom &g = a.g;
    const Model &m = a.m;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x >= g.nx)
            continue;
        const int o = y * g.pitch + x;
        const float S0 = a.S0[o];
        const float sx = fd_axis(a.S0, g, x, y, 0), sy = fd_axis(a.S0, g, x, y, 1);
        float f[8];
        gather_a(a.fin, a.R, g, a.Pb, x, y, o, f);
        a.Pnew[o] = a.R[o] + pressure_of(f);
        float mx, my;
        first_moment(f, mx, my);
        const float it = a.inv_tau[o];
        const float gx = -3.0f * mx * it, gy = -3.0f * my * it;
        const float Fs = saturation_source(m, a.w, a.Fs, o, S0);   // S* = S0 at t = 0
        const float K = a.K[o];
        float lw, lt;
        mobility(m, S0, lw, lt);
        float inv_tg0, src_g0;
        tau_g_node(m, K, lw, lt, inv_tg0, src_g0);
        const float tg = 1.0f / inv_tg0;
        const float gam0 = -m.gam_c * lw * K;
        float q[9];
        float sum = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            q[i] = 0.0f;
            if (i >= m.qs)
                continue;
            const float wi = m.wg[i];
            const float cS = (float)cx(i) * sx + (float)cy(i) * sy;
            const float cP = (float)cx(i) * gx + (float)cy(i) * gy;
            const float neq = -tg * ((m.Gam[i] * m.inv_phi - wi * src_g0) * Fs + m.Gam[i] * cS
                                     - gam0 * wi * cP * inv_tg0);
            q[i] = m.Gam[i] * S0 + neq;
            sum += q[i];
        }
        const float S = (sum + 0.5f * Fs) * m.inv_phi;
        mobility(m, S, lw, lt);
        float inv_tg, src_g;
        tau_g_node(m, K, lw, lt, inv_tg, src_g);
        const float gam = -m.gam_c * lw * K * inv_tg;
        const float src = src_g * Fs;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i >= m.qs)
                break;
            const float wi = m.wg[i];
            const float cg = (float)cx(i) * gx + (float)cy(i) * gy;
            a.gout[i][o] = fmaf(m.Gam[i] * S - q[i], inv_tg, q[i]) + wi * src + gam * wi * cg;
        }
        a.S[o] = S;
    }
}

// Four nodes per thread with 128-bit accesses (rows are padded to 32 floats, so a quad never
// crosses a row); per node the arithmetic of rebase_node.  Padding lanes are written back
// unchanged.
__global__ void __launch_bounds__(kBlock) k_rebase(const __grid_constant__ RebaseArgs a)
{
    const Geom &g = a.g;
    const int qx = (g.nx + 3) / 4;
    const long long nq = (long long)qx * g.ny;
    for (long long q = (long long)blockIdx.x * kBlock + threadIdx.x; q < nq;
         q += (long long)gridDim.x * kBlock) {
        const int y = (int)(q / qx);
        const int x = (int)(q - (long long)y * qx) * 4;
        const int o = y * g.pitch + x;
        const float4 r = *reinterpret_cast<const float4 *>(a.R + o);
        const float4 pn = *reinterpret_cast<const float4 *>(a.Pnew + o);
        const bool in1 = x + 1 < g.nx, in2 = x + 2 < g.nx, in3 = x + 3 < g.nx;
        float4 d;
        d.x = r.x - pn.x;
        d.y = in1 ? r.y - pn.y : 0.0f;
        d.z = in2 ? r.z - pn.z : 0.0f;
        d.w = in3 ? r.w - pn.w : 0.0f;
        float4 n[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            n[i] = *reinterpret_cast<const float4 *>(a.n[i] + o);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float w = wgt(i + 1);
            float4 v = n[i];
            v.x = fmaf(w, d.x, v.x);
            if (in1)
                v.y = fmaf(w, d.y, v.y);
            if (in2)
                v.z = fmaf(w, d.z, v.z);
            if (in3)
                v.w = fmaf(w, d.w, v.w);
            *reinterpret_cast<float4 *>(a.n[i] + o) = v;
        }
        float4 rn = r;
        rn.x = pn.x;
        if (in1)
            rn.y = pn.y;
        if (in2)
            rn.z = pn.z;
        if (in3)
            rn.w = pn.w;
        *reinterpret_cast<float4 *>(a.R + o) = rn;
    }
}

__global__ void __launch_bounds__(kBlock) k_rebase_mid(const __grid_constant__ RebaseMidArgs a)
{
    const Geom &g = a.g;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx)
            rebase_mid_node(a, y * g.pitch + x);
    }
}

__global__ void __launch_bounds__(kBlock) k_tau_from_S(float *inv_tau, const float *S,
                                                       const float *K, Geom g, Model m)
{
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x >= g.nx)
            continue;
        const int o = y * g.pitch + x;
        float lw, lt;
        mobility(m, S[o], lw, lt);
        inv_tau[o] = 1.0f / (0.5f + m.s3 * K[o] * lt);
    }
}

// --------------------------------------------------------------------------------------
// fields: P (Eq. 3-9a), S, u = -K lambda_t grad P (Eq. 3-10b) into compact [ny][nx]
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_fields(const __grid_constant__ FieldsArgs a)
{
    const Geom &g = a.g;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x >= g.nx)
            continue;
        const int o = y * g.pitch + x;
        const long long c = (long long)y * g.nx + x;
        float f[8];
        gather_a(a.fin, a.R, g, a.Pb, x, y, o, f);
        const float S = a.S[o];
        if (a.P_out)
            a.P_out[c] = a.R[o] + pressure_of(f);
        if (a.S_out)
            a.S_out[c] = S;
        if (a.ux_out || a.uy_out) {
            float mx, my;
            first_moment(f, mx, my);
            const float it = a.inv_tau[o];
            const float gpx = -3.0f * mx * it * a.m.inv_dx, gpy = -3.0f * my * it * a.m.inv_dx;
            float lw, lt;
            mobility(a.m, S, lw, lt);
            const float kl = a.K[o] * lt;
            if (a.ux_out)
                a.ux_out[c] = -kl * gpx;
            if (a.uy_out)
                a.uy_out[c] = -kl * gpy;
        }
    }
}

__global__ void __launch_bounds__(256) k_sum_compact(const float *__restrict__ x, long long n,
                                                     double *partials)
{
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x)
        s += (double)x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        partials[blockIdx.x] = red[0];
}

__global__ void k_finalize_mean(const double *partials, int nparts, long long n, double *mean)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nparts; ++i)
            s += partials[i];
        *mean = s / (double)n;
    }
}

__global__ void __launch_bounds__(256) k_subtract_mean(float *x, long long n, const double *mean)
{
    const float m = (float)*mean;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x)
        x[i] -= m;
}

}  // namespace lbm2p_dev

// ======================================================================================
// launchers
// ======================================================================================
namespace lbm2p_launch {

static cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static void *sweep_func(int kind, bool check, bool write_p)
{
    if (kind == 1)
        return check ? (write_p ? (void *)k_pressure_scalar<true, true> : (void *)k_pressure_scalar<true, false>)
                     : (write_p ? (void *)k_pressure_scalar<false, true> : (void *)k_pressure_scalar<false, false>);
    return check ? (write_p ? (void *)k_pressure<true, true> : (void *)k_pressure<true, false>)
                 : (write_p ? (void *)k_pressure<false, true> : (void *)k_pressure<false, false>);
}

int max_blocks_per_sm_pressure(bool check, int kind)
{
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, sweep_func(kind, check, true), kBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_func(kind, check, false), kBlock, 0);
    int m = a < b ? a : b;
    return m > 0 ? m : 1;
}

void pressure_sweep(const PressureArgs &a, bool check, bool write_p, int grid, void *stream,
                    int kind)
{
    // grid: resident capacity of the chosen kernel; check sweeps use the capacity of theirs
    void *args[] = {(void *)&a};
    cudaLaunchKernel(sweep_func(kind, check, write_p), dim3(grid), dim3(kBlock), args, 0, S(stream));
}

size_t tb_smem_bytes(int T, int Wt)
{
    size_t floats = 0;
    for (int s = 0; s < T; ++s)
        floats += 24 * (size_t)(Wt - 2 * s);
    floats += 3 * (size_t)(T + 2) * Wt + 3 * (size_t)(Wt - 2 * T + 2);
    return floats * sizeof(float);
}

long long tb_grid(int T, int Wt, int H, int nx, int ny)
{
    const int W = Wt - 2 * T;
    return (long long)((nx + W - 1) / W) * ((ny + H - 1) / H);
}

static void *tb_func(int T, bool check)
{
    if (T == 2)
        return check ? (void *)k_pressure_tb<2, true> : (void *)k_pressure_tb<2, false>;
    return check ? (void *)k_pressure_tb<4, true> : (void *)k_pressure_tb<4, false>;
}

cudaError_t tb_prepare(int T, int W)
{
    // the opt-in limit is set for the widest tile, so every tile width stays launchable
    const int bytes = (int)tb_smem_bytes(T, W > 128 ? W : 128);
    cudaError_t e = cudaSuccess;
    for (bool c : {false, true}) {
        e = cudaFuncSetAttribute(tb_func(T, c), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    return e;
}

int tb_blocks_per_sm(int T, int W)
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tb_func(T, true), W, tb_smem_bytes(T, W));
    return b;
}

void pressure_sweeps_fused(const PressureArgs &a, int T, int W, int H, bool check, int grid,
                           void *stream)
{
    void *args[] = {(void *)&a, (void *)&H};
    cudaLaunchKernel(tb_func(T, check), dim3(grid), dim3(W), args, tb_smem_bytes(T, W), S(stream));
}

void residual_finalize(const double *partials, int nparts, long long nnodes, float *shift,
                       ResidualOut *out, void *stream)
{
    k_residual_finalize<<<1, 256, 0, S(stream)>>>(partials, nparts, nnodes, shift, out);
}

void refresh(const RefreshArgs &a, int grid, void *stream)
{
    k_refresh<<<grid, kBlock, 0, S(stream)>>>(a);
}

void saturation(const SaturationArgs &a, int grid, void *stream)
{
    k_saturation<<<grid, kBlock, 0, S(stream)>>>(a);
}

void init_g(const InitGArgs &a, int grid, void *stream)
{
    k_init_g<<<grid, kBlock, 0, S(stream)>>>(a);
}

void rebase(const RebaseArgs &a, int grid, void *stream)
{
    k_rebase<<<grid, kBlock, 0, S(stream)>>>(a);
}

void rebase_mid(const RebaseMidArgs &a, int grid, void *stream)
{
    k_rebase_mid<<<grid, kBlock, 0, S(stream)>>>(a);
}

void tau_from_S(float *inv_tau, const float *Sp, const float *K, Geom g, Model m, int grid,
                void *stream)
{
    k_tau_from_S<<<grid, kBlock, 0, S(stream)>>>(inv_tau, Sp, K, g, m);
}

void fields(const FieldsArgs &a, int grid, void *stream)
{
    k_fields<<<grid, kBlock, 0, S(stream)>>>(a);
}

void sum_compact(const float *x, long long n, double *partials, int grid, void *stream)
{
    k_sum_compact<<<grid, 256, 0, S(stream)>>>(x, n, partials);
}

void finalize_mean(const double *partials, int nparts, long long n, double *mean, void *stream)
{
    k_finalize_mean<<<1, 32, 0, S(stream)>>>(partials, nparts, n, mean);
}

void subtract_mean(float *x, long long n, const double *mean, int grid, void *stream)
{
    k_subtract_mean<<<grid, 256, 0, S(stream)>>>(x, n, mean);
}

static cudaError_t add_kernel(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                              void *func, int grid, int block, void **args)
{
    cudaKernelNodeParams p{};
    p.func = func;
    p.gridDim = dim3((unsigned)grid);
    p.blockDim = dim3((unsigned)block);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    p.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &p);
}

cudaError_t node_pressure(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                          const PressureArgs &a, bool check, bool write_p, int grid, int kind)
{
    void *args[] = {(void *)&a};
    return add_kernel(n, g, dep, sweep_func(kind, check, write_p), grid, kBlock, args);
}

cudaError_t node_pressure_fused(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                                const PressureArgs &a, int T, int W, int H, bool check, int grid)
{
    cudaKernelNodeParams p{};
    p.func = tb_func(T, check);
    p.gridDim = dim3((unsigned)grid);
    p.blockDim = dim3((unsigned)W);
    p.sharedMemBytes = (unsigned)tb_smem_bytes(T, W);
    void *args[] = {(void *)&a, (void *)&H};
    p.kernelParams = args;
    p.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &p);
}

cudaError_t node_finalize_loop(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                               const double *partials, int nparts, long long nnodes, float *shift,
                               ResidualOut *out, LoopCtl *ctl, cudaGraphConditionalHandle h,
                               cudaGraphConditionalHandle h_rebase)
{
    void *args[] = {(void *)&partials, (void *)&nparts, (void *)&nnodes, (void *)&shift,
                    (void *)&out, (void *)&ctl, (void *)&h, (void *)&h_rebase};
    return add_kernel(n, g, dep, (void *)k_residual_finalize_loop, 1, 256, args);
}

cudaError_t node_rebase_mid(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            const RebaseMidArgs &a, int grid)
{
    void *args[] = {(void *)&a};
    return add_kernel(n, g, dep, (void *)k_rebase_mid, grid, kBlock, args);
}

cudaError_t node_loop_reset(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            LoopCtl *ctl)
{
    void *args[] = {(void *)&ctl};
    return add_kernel(n, g, dep, (void *)k_loop_reset, 1, 1, args);
}

cudaError_t node_if_finite(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                           const LoopCtl *ctl, cudaGraphConditionalHandle h)
{
    void *args[] = {(void *)&ctl, (void *)&h};
    return add_kernel(n, g, dep, (void *)k_if_finite, 1, 1, args);
}

cudaError_t node_refresh(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                         const RefreshArgs &a, int grid)
{
    void *args[] = {(void *)&a};
    return add_kernel(n, g, dep, (void *)k_refresh, grid, kBlock, args);
}

cudaError_t node_saturation(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            const SaturationArgs &a, int grid)
{
    void *args[] = {(void *)&a};
    return add_kernel(n, g, dep, (void *)k_saturation, grid, kBlock, args);
}

cudaError_t node_rebase(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                        const RebaseArgs &a, int grid)
{
    void *args[] = {(void *)&a};
    return add_kernel(n, g, dep, (void *)k_rebase, grid, kBlock, args);
}

}  // namespace lbm2p_launch
