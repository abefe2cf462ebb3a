// Device functions of one lattice node, shared by every kernel of the solver: the
// gathers with the wall rules of Sec. 4, the per-node arithmetic of the two LBEs, and the
// per-node bodies of the single-lattice and batched kernels (so both compute bit for bit
// the same values).
#pragma once

#include "lbm2p_device.cuh"

namespace lbm2p_dev {

// --------------------------------------------------------------------------------------
// gather with the wall rules of Sec. 4
// --------------------------------------------------------------------------------------
// The per-node arithmetic of a pressure sweep, written with explicit fused multiply-adds so
// that every kernel that performs a sweep (one per launch, or several fused in one launch)
// produces bit-identical populations.
// a_i = n_i(src) + w_i (R(src) - R(x))
__device__ __forceinline__ float dev1(float n, float w, float r, float r0)
{
    return fmaf(w, r - r0, n);
}

// n_i^+ = a_i + (w_i dP - a_i) / tau_f + F~_p / 8   (Eq. 2-1b relative to R)
__device__ __forceinline__ float collide1(float a, float w, float dP, float it, float Fq)
{
    return fmaf(fmaf(w, dP, -a), it, a) + Fq;
}

__device__ __forceinline__ bool interior(const Geom &g, int x, int y)
{
    return x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1;
}

// a_I = f_I(x) - w_I R(x) pulled into an edge node (x, y), with r0 = R(x).  Wall rules of
// Sec. 4 in deviation form: a neighbour inside (or wrapped) gives n_I(src) + w_I (R(src) - r0);
// bounce-back gives n_opp(x); anti-bounce-back gives -n_opp(x) + 2 w_I (P_b - r0).
template <int I>
__device__ __forceinline__ float pull_edge_dev(const float *__restrict__ n_i,
                                               const float *__restrict__ n_opp,
                                               const float *__restrict__ R, const Geom &g,
                                               const float *const *Pb, int x, int y, float r0)
{
    constexpr int ex = cx(I), ey = cy(I);
    int xs = x - ex, ys = y - ey, side = -1;
    if (xs < 0 || xs >= g.nx) {
        const int sd = xs < 0 ? 0 : 1;
        if (g.bc[sd] == BC_PERIODIC)
            xs += xs < 0 ? g.nx : -g.nx;
        else
            side = sd;
    }
    if (side < 0 && (ys < 0 || ys >= g.ny)) {
        const int sd = ys < 0 ? 2 : 3;
        if (g.bc[sd] == BC_PERIODIC)
            ys += ys < 0 ? g.ny : -g.ny;
        else
            side = sd;
    }
    if (side < 0) {
        const int src = ys * g.pitch + xs;
        return dev1(n_i[src], wgt(I), R[src], r0);
    }
    const float b = n_opp[y * g.pitch + x];
    if (g.bc[side] == BC_NOFLUX)
        return b;
    const int k = side < 2 ? 2 * y + 1 - ey : 2 * x + 1 - ex;
    return -b + 2.0f * wgt(I) * (Pb[side][k] - r0);
}

// a_1 .. a_8 (pressure populations relative to R(x)) pulled into (x, y)
__device__ __forceinline__ void gather_a(const float *const *fin, const float *__restrict__ R,
                                         const Geom &g, const float *const *Pb, int x, int y,
                                         int o, float (&a)[8])
{
    const float r0 = R[o];
    if (interior(g, x, y)) {
        const int p = g.pitch;
        a[0] = dev1(fin[0][o - 1], wgt(1), R[o - 1], r0);
        a[1] = dev1(fin[1][o - p], wgt(2), R[o - p], r0);
        a[2] = dev1(fin[2][o + 1], wgt(3), R[o + 1], r0);
        a[3] = dev1(fin[3][o + p], wgt(4), R[o + p], r0);
        a[4] = dev1(fin[4][o - p - 1], wgt(5), R[o - p - 1], r0);
        a[5] = dev1(fin[5][o - p + 1], wgt(6), R[o - p + 1], r0);
        a[6] = dev1(fin[6][o + p + 1], wgt(7), R[o + p + 1], r0);
        a[7] = dev1(fin[7][o + p - 1], wgt(8), R[o + p - 1], r0);
    } else {
        a[0] = pull_edge_dev<1>(fin[0], fin[opp(1) - 1], R, g, Pb, x, y, r0);
        a[1] = pull_edge_dev<2>(fin[1], fin[opp(2) - 1], R, g, Pb, x, y, r0);
        a[2] = pull_edge_dev<3>(fin[2], fin[opp(3) - 1], R, g, Pb, x, y, r0);
        a[3] = pull_edge_dev<4>(fin[3], fin[opp(4) - 1], R, g, Pb, x, y, r0);
        a[4] = pull_edge_dev<5>(fin[4], fin[opp(5) - 1], R, g, Pb, x, y, r0);
        a[5] = pull_edge_dev<6>(fin[5], fin[opp(6) - 1], R, g, Pb, x, y, r0);
        a[6] = pull_edge_dev<7>(fin[6], fin[opp(7) - 1], R, g, Pb, x, y, r0);
        a[7] = pull_edge_dev<8>(fin[7], fin[opp(8) - 1], R, g, Pb, x, y, r0);
    }
}

// generic pull for the saturation populations (plain values, planes 0..8)
template <int I>
__device__ __forceinline__ float pull_edge(const float *__restrict__ src_i,
                                           const float *__restrict__ src_opp, const Geom &g,
                                           const float *const *trace, float eq_opp, int x,
                                           int y)
{
    constexpr int ex = cx(I), ey = cy(I);
    int xs = x - ex, ys = y - ey, side = -1;
    if (xs < 0 || xs >= g.nx) {
        const int sd = xs < 0 ? 0 : 1;
        if (g.bc[sd] == BC_PERIODIC)
            xs += xs < 0 ? g.nx : -g.nx;
        else
            side = sd;
    }
    if (side < 0 && (ys < 0 || ys >= g.ny)) {
        const int sd = ys < 0 ? 2 : 3;
        if (g.bc[sd] == BC_PERIODIC)
            ys += ys < 0 ? g.ny : -g.ny;
        else
            side = sd;
    }
    if (side < 0)
        return src_i[ys * g.pitch + xs];
    const float b = src_opp[y * g.pitch + x];
    if (g.bc[side] == BC_NOFLUX)
        return b;
    const int k = side < 2 ? 2 * y + 1 - ey : 2 * x + 1 - ex;
    return -b + 2.0f * eq_opp * trace[side][k];
}

// g_0 .. g_8 pulled into (x, y) (saturation distribution, planes 0..8)
__device__ __forceinline__ void gather_g(const float *const *gin, const Geom &g, const Model &m,
                                         const float *const *Sb, int x, int y, int o,
                                         float (&q)[9])
{
    // D2Q5 (m.qs == 5) carries populations 0..4 only; the diagonal slots read as zero
    q[0] = gin[0][o];
    q[5] = q[6] = q[7] = q[8] = 0.0f;
    if (interior(g, x, y)) {
        const int p = g.pitch;
        q[1] = gin[1][o - 1];
        q[2] = gin[2][o - p];
        q[3] = gin[3][o + 1];
        q[4] = gin[4][o + p];
        if (m.qs == 9) {
            q[5] = gin[5][o - p - 1];
            q[6] = gin[6][o - p + 1];
            q[7] = gin[7][o + p + 1];
            q[8] = gin[8][o + p - 1];
        }
    } else {
        q[1] = pull_edge<1>(gin[1], gin[opp(1)], g, Sb, m.Gam[opp(1)], x, y);
        q[2] = pull_edge<2>(gin[2], gin[opp(2)], g, Sb, m.Gam[opp(2)], x, y);
        q[3] = pull_edge<3>(gin[3], gin[opp(3)], g, Sb, m.Gam[opp(3)], x, y);
        q[4] = pull_edge<4>(gin[4], gin[opp(4)], g, Sb, m.Gam[opp(4)], x, y);
        if (m.qs == 9) {
            q[5] = pull_edge<5>(gin[5], gin[opp(5)], g, Sb, m.Gam[opp(5)], x, y);
            q[6] = pull_edge<6>(gin[6], gin[opp(6)], g, Sb, m.Gam[opp(6)], x, y);
            q[7] = pull_edge<7>(gin[7], gin[opp(7)], g, Sb, m.Gam[opp(7)], x, y);
            q[8] = pull_edge<8>(gin[8], gin[opp(8)], g, Sb, m.Gam[opp(8)], x, y);
        }
    }
}

// 1/tau_g and 1 - 1/(2 tau_g) at a node: constants when D_s is constant, otherwise
// tau_g = 1/2 + 3 D_s(x, S) dt / (beta dx^2) with D_s = D_s + D_c K lambda_w lambda_n /
// lambda_t (Eq. 3-11b with the diffusivity of Eq. 2-16 for a linear capillary pressure)
__device__ __forceinline__ void tau_g_node(const Model &m, float K, float lw, float lt,
                                           float &inv_tg, float &src)
{
    if (!m.var_ds) {
        inv_tg = m.inv_tau_g;
        src = m.src_g;
        return;
    }
    const float h = lt != 0.0f ? lw * (lt - lw) / lt : 0.0f;
    inv_tg = 1.0f / (0.5f + m.ds_a0 + m.ds_a1 * K * h);
    src = 1.0f - 0.5f * inv_tg;
}

// Eq. 3-9a: P = sum_{i=1..8} f_i / (1 - w_0) = (9/5) sum
__device__ __forceinline__ float pressure_of(const float (&f)[8])
{
    return (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) * 1.8f;
}

// sum_i c_i f_i (x and y components)
__device__ __forceinline__ void first_moment(const float (&f)[8], float &mx, float &my)
{
    mx = (f[0] - f[2]) + ((f[4] - f[5]) - (f[6] - f[7]));
    my = (f[1] - f[3]) + ((f[4] + f[5]) - (f[6] + f[7]));
}

__device__ __forceinline__ void mobility(const Model &m, float S, float &lw, float &lt)
{
    if (m.mobility == MOB_QUADRATIC) {
        lw = S * S * m.inv_mu_w;
        const float sn = 1.0f - S;
        lt = lw + sn * sn * m.inv_mu_n;
    } else if (m.mobility == MOB_DECOUPLED) {
        lw = m.inv_mu_w;
        lt = m.inv_mu_w;
    } else {
        lt = 1.0f / (0.5f - 0.2f * S);
        lw = S * lt;
    }
}

// dt F_s at node o: dense part plus wells; the producer uses S* = sum g / phi.
__device__ __forceinline__ float saturation_source(const Model &m, const Wells &w,
                                                   const float *Fs, int o, float Sstar)
{
    float F = Fs ? Fs[o] : 0.0f;
    for (int k = 0; k < w.n; ++k) {
        if (o == w.idx[k]) {
            if (w.producer[k]) {
                float lw, lt;
                mobility(m, Sstar, lw, lt);
                F -= w.qs[k] * (lt != 0.0f ? lw / lt : 0.0f);
            } else {
                F += w.qs[k];
            }
        }
    }
    return F;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int s = 16; s > 0; s >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// Residual sums of a checking sweep (a3): sum d, sum d^2, sum q, sum q^2 over the nodes of a
// warp, accurate whatever the shift constants already subtracted from d and q.  Each thread
// sums in FP32 the differences of its values from the first ones it saw (its pivots), which
// are of the size of the spread of d and q, not of their offset; at the end the lanes move
// their sums to the pivots of the warp's lowest active lane (again a difference of two
// samples), the warp adds them in FP32, and lane 0 restores the raw sums in FP64:
// sum x = S1 + n c, sum x^2 = S2 + 2 c S1 + n c^2.
struct ResAcc {
    int n = 0;
    float cd = 0.0f, cq = 0.0f;                    // pivots of this thread
    float s1 = 0.0f, s2 = 0.0f, t1 = 0.0f, t2 = 0.0f;

    __device__ __forceinline__ void add(float d, float q)
    {
        if (n == 0) {
            cd = d;
            cq = q;
        }
        const float e = d - cd, u = q - cq;
        s1 += e;
        s2 = fmaf(e, e, s2);
        t1 += u;
        t2 = fmaf(u, u, t2);
        ++n;
    }

    // called by all 32 lanes together; lane 0 receives the warp's raw sums
    __device__ __forceinline__ void warp_totals(double (&v)[4]) const
    {
        const unsigned act = __ballot_sync(0xffffffffu, n > 0);
        const int src = act ? __ffs(act) - 1 : 0;
        const float wd = __shfl_sync(0xffffffffu, cd, src);
        const float wq = __shfl_sync(0xffffffffu, cq, src);
        const float nf = (float)n;
        float a1 = 0.0f, a2 = 0.0f, b1 = 0.0f, b2 = 0.0f;
        if (n > 0) {
            const float od = cd - wd, oq = cq - wq;  // this thread's pivots from the warp's
            a1 = fmaf(nf, od, s1);
            a2 = fmaf(nf * od, od, fmaf(2.0f * od, s1, s2));
            b1 = fmaf(nf, oq, t1);
            b2 = fmaf(nf * oq, oq, fmaf(2.0f * oq, t1, t2));
        }
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
        b1 = warp_sum(b1);
        b2 = warp_sum(b2);
        int cnt = n;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1)
            cnt += __shfl_xor_sync(0xffffffffu, cnt, sh);
        if ((threadIdx.x & 31) == 0) {
            const double N = (double)cnt, c = (double)wd, b = (double)wq;
            v[0] = (double)a1 + N * c;
            v[1] = (double)a2 + 2.0 * c * (double)a1 + N * c * c;
            v[2] = (double)b1 + N * b;
            v[3] = (double)b2 + 2.0 * b * (double)b1 + N * b * b;
        }
    }
};


// --------------------------------------------------------------------------------------
// per-node bodies shared by the single-lattice kernels and the batched kernels
// --------------------------------------------------------------------------------------
// Warm start of a solve: the equilibrium part of f_i = n_i + w_i R moves with R to the
// pressure extrapolated in time, R' = R + (R - P^{n-1}); n_i (the rest) is kept.  The inputs
// may be the outputs (in place).
__device__ __forceinline__ void extrapolate_node(const float *Rin, float *Rout,
                                                 const float *Pin, float *Pout, int o)
{
    const float r = Rin[o];
    const float pv = Pin[o];
    Rout[o] = r + (r - pv);
    Pout[o] = r;
}

// a1: S^n (Eq. 3-9b) from the pulled g and 1/tau_f (Eq. 3-11a with D_p = K lambda_t(S)); with
// a warm start also the extrapolation of the node's reference pressure for the coming solve
__device__ __forceinline__ void refresh_node(const RefreshArgs &a, int x, int y, int o)
{
    float q[9];
    gather_g(a.gin, a.g, a.m, a.Sb, x, y, o, q);
    const float sum = (q[0] + ((q[1] + q[2]) + (q[3] + q[4]))) + ((q[5] + q[6]) + (q[7] + q[8]));
    const float Fs = saturation_source(a.m, a.w, a.Fs, o, sum * a.m.inv_phi);
    const float S = (sum + 0.5f * Fs) * a.m.inv_phi;
    float lw, lt;
    mobility(a.m, S, lw, lt);
    a.inv_tau[o] = 1.0f / (0.5f + a.m.s3 * a.K[o] * lt);
    if (a.Pstep_in)
        extrapolate_node(a.Rin, a.Rout, a.Pstep_in, a.Pstep_out, o);
    else if (a.Rout != a.Rin)
        a.Rout[o] = a.Rin[o];
}

// a4 + a5: local grad P (Eq. 3-10a), then the saturation collision (Eq. 3-2); also stores
// S^n and the pressure of the pulled state (for the rebase)
__device__ __forceinline__ void saturation_node(const SaturationArgs &a, int x, int y, int o)
{
    const Geom &g = a.g;
    const Model &m = a.m;
    float f[8], q[9];
    gather_a(a.fin, a.R, g, a.Pb, x, y, o, f);
    a.Pnew[o] = a.R[o] + pressure_of(f);
    gather_g(a.gin, g, m, a.Sb, x, y, o, q);
    const float sum = (q[0] + ((q[1] + q[2]) + (q[3] + q[4]))) + ((q[5] + q[6]) + (q[7] + q[8]));
    const float Fs = saturation_source(m, a.w, a.Fs, o, sum * m.inv_phi);
    const float S = (sum + 0.5f * Fs) * m.inv_phi;
    // grad_X P = -3 sum_i c_i f_i / tau_f  (lattice units, Eq. 3-10a)
    float mx, my;
    first_moment(f, mx, my);
    const float it = a.inv_tau[o];
    const float gx = -3.0f * mx * it, gy = -3.0f * my * it;
    float lw, lt;
    mobility(m, S, lw, lt);
    const float K = a.K[o];
    float inv_tg, src_g;
    tau_g_node(m, K, lw, lt, inv_tg, src_g);
    // gamma~ = -3 lambda_w K dt / dx^2 (Eq. 3-8 in lattice units), pre-divided by tau_g
    const float gam = -m.gam_c * lw * K * inv_tg;
    const float src = src_g * Fs;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (i >= m.qs)
            break;
        const float wi = m.wg[i];
        const float cg = (float)cx(i) * gx + (float)cy(i) * gy;
        const float eq = m.Gam[i] * S;
        a.gout[i][o] = fmaf(eq - q[i], inv_tg, q[i]) + wi * src + gam * wi * cg;
    }
    a.S[o] = S;
}

// move the reference pressure to Pnew: n_i += w_i (R - Pnew), R = Pnew (own node only)
__device__ __forceinline__ void rebase_node(const RebaseArgs &a, int o)
{
    const float pn = a.Pnew[o];
    const float d = a.R[o] - pn;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        a.n[i][o] = fmaf(wgt(i + 1), d, a.n[i][o]);
    a.R[o] = pn;
}

// Within a long sub-iteration, move R to the current pressure.  After a sweep the stored
// populations satisfy sum_{i>=1} n_i^+ = (5/9) dP + F~_p (the collision of Eq. 2-1b summed
// over i >= 1, sum w_i = 5/9), so dP = (9/5)(sum_i n_i^+ - F~_p) is the node's increment
// over R.  n_i -= w_i dP, R += dP leaves every f_i = n_i + w_i R unchanged (any new R is
// exact); it keeps the deviations, and so their FP32 rounding, small.
__device__ __forceinline__ void rebase_mid_node(const RebaseMidArgs &a, int o)
{
    float F = a.Fp ? a.Fp[o] : 0.0f;
    for (int k = 0; k < a.w.n; ++k)
        if (o == a.w.idx[k])
            F += a.w.fp[k];
    float n[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        n[i] = a.n[i][o];
    const float dP = 1.8f * ((((n[0] + n[1]) + (n[2] + n[3])) + ((n[4] + n[5]) + (n[6] + n[7]))) - F);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        a.n[i][o] = fmaf(-wgt(i + 1), dP, n[i]);
    a.R[o] = a.R[o] + dP;
}

// a2: one node of a pressure sweep with scalar gathers; (d, q) feed the residual partials
template <bool CHECK, bool WRITE_P>
__device__ __forceinline__ void sweep_node(const PressureArgs &a, int x, int y, int o,
                                           float shift, float dshift, float &d, float &q)
{
    float f[8];
    gather_a(a.fin, a.R, a.g, a.Pb, x, y, o, f);
    const float dP = pressure_of(f);
    const float it = a.inv_tau[o];
    float F = a.Fp ? a.Fp[o] : 0.0f;
    for (int k = 0; k < a.w.n; ++k)
        if (o == a.w.idx[k])
            F += a.w.fp[k];
    const float Fq = 0.125f * F;   // w_bar_i = 1/8 (Eq. 3-5a)
#pragma unroll
    for (int i = 0; i < 8; ++i)
        a.fout[i][o] = collide1(f[i], wgt(i + 1), dP, it, Fq);
    if (CHECK) {
        d = (dP - a.Pio[o]) - dshift;
        q = (a.R[o] - shift) + dP;
    }
    if (WRITE_P)
        a.Pio[o] = dP;
}

}  // namespace lbm2p_dev
