// Pressure sweep (Eq. 3-1, pull stream + BGK collide) with its input rows staged in shared
// memory by the bulk-copy engine.
//
// A block owns a strip of W columns and a chunk of H rows, and marches down the chunk.  Pulling into row y reads populations of rows y-1 (directions with c_y = +1),
// y (c_y = 0) and y+1 (c_y = -1), the reference pressure R of all three rows, and 1/tau_f
// and F~_p of row y.  Each input row r is therefore copied once, as row segments
// [x0 - 4, x0 + W + 4) of every plane (16-byte aligned, clamped to the row), by one
// cp.async.bulk per plane into a ring of S slots by a producer warp, while consumer warps
// compute; full/empty mbarriers per slot hand rows between them.  The
// arithmetic of an interior node is that of gather_a / sweep_node with the loads taken
// from shared memory; edge nodes take the global-memory gather with the wall rules.  The
// populations written are bit-identical to the other single-sweep kernels.
//
// Every wait on an mbarrier is bounded: a block that gives up waits (bounded) for its own
// copies still in flight, writes NaN into its outputs and residual partials, and returns,
// so the host sees a non-finite residual instead of a hung GPU.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm2p_async.cuh"
#include "lbm2p_device.cuh"
#include "lbm2p_node.cuh"

namespace lbm2p_dev {
namespace {

constexpr int kRowsMaxPlanes = 11;            // n_1..n_8, R, 1/tau_f, F~_p (when present)
constexpr int kRowsHalo = 4;                  // floats staged on each side of the strip
constexpr int kRowsBarBytes = 128;            // mbarriers at the start of shared memory

// Warp-specialised pipeline.  Warp CW is the producer: its lane 0 copies input row t into
// slot t % S once the consumers have released the row that used it before (row t - S).
// Warps 0 .. CW-1 are consumers, each owning 32 columns of the strip: a consumer waits for
// row t (full barrier), computes output row t - 1 from rows t - 2 .. t, and releases row
// t - 2 (empty barrier, one arrival per consumer warp).  No block-wide barrier per row.
template <bool CHECK, bool WRITE_P, int CW, int S>
__global__ void __launch_bounds__(32 * (CW + 1)) k_pressure_rows(const __grid_constant__ PressureArgs a,
                                                                 int H)
{
    constexpr int W = 32 * CW;
    constexpr int RW = W + 2 * kRowsHalo;          // floats per staged plane row
    const int npl = a.Fp ? 11 : 10;                // planes staged per row
    const int slot_floats = npl * RW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk copies need 16-byte aligned destinations: align the ring explicitly (the launch
    // adds 128 bytes of slack for this)
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + S;
    float *ring = reinterpret_cast<float *>(smem + kRowsBarBytes);
    __shared__ double red[CW][4];
    __shared__ int failed;
    const Geom &g = a.g;
    const int p = g.pitch;
    const int strips = (g.nx + W - 1) / W;
    const int x0 = (blockIdx.x % strips) * W;
    const int y0 = (blockIdx.x / strips) * H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (y0 >= g.ny) {                              // not produced by rows_grid; kept safe
        if (CHECK && threadIdx.x < 4)
            a.partials[4 * blockIdx.x + threadIdx.x] = 0.0;
        return;
    }
    const int y1 = y0 + H < g.ny ? y0 + H : g.ny;
    const int nrows = y1 - y0 + 2;                 // input rows y0 - 1 .. y1
    // segment of every staged row: [xa, xb) in the plane, at xa - (x0 - halo) in the slot
    const int xa = x0 - kRowsHalo > 0 ? x0 - kRowsHalo : 0;
    const int xb = x0 + W + kRowsHalo < p ? x0 + W + kRowsHalo : p;
    const unsigned seg = (unsigned)(xb - xa) * 4u;
    const int soff = xa - (x0 - kRowsHalo);

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            bar_init(full + q, 1);
            bar_init(empty + q, CW);
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == CW) {
        // ---- producer ------------------------------------------------------------------
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nrows; ++t) {
                const int q = t % S;
                if (t >= S && !bar_wait_bounded(empty + q, (unsigned)(t / S - 1) & 1u)) {
                    failed = 1;
                    break;
                }
                // planes of input row t (y0 - 1 + t): the first row feeds only the c_y = +1
                // pulls of row y0, the last only the c_y = -1 pulls of row y1 - 1; both
                // also give R
                const int r = y0 - 1 + t;
                unsigned m = npl == 11 ? 0x7FFu : 0x3FFu;
                if (r < 0 || r >= g.ny)
                    m = 0u;
                else if (t == 0)
                    m = (1u << 1) | (1u << 4) | (1u << 5) | (1u << 8);
                else if (t == nrows - 1)
                    m = (1u << 3) | (1u << 6) | (1u << 7) | (1u << 8);
                if (!m) {
                    bar_arrive(full + q);
                } else {
                    bar_arrive_tx(full + q, (unsigned)__popc(m) * seg);
                    const size_t roff = (size_t)r * p + xa;
                    float *slot = ring + (size_t)q * slot_floats + soff;
#pragma unroll
                    for (int pl = 0; pl < kRowsMaxPlanes; ++pl) {
                        if (!(m & (1u << pl)))
                            continue;
                        const float *src = pl < 8 ? a.fin[pl]
                                                  : (pl == 8 ? a.R : (pl == 9 ? a.inv_tau : a.Fp));
                        bulk_g2s(slot + pl * RW, src + roff, seg, full + q);
                    }
                }
                issued = t + 1;
            }
            // no copy may still be landing in this block's shared memory when it exits
            for (int t = issued - S > 0 ? issued - S : 0; t < issued; ++t)
                bar_wait_bounded(full + t % S, (unsigned)(t / S) & 1u);
        }
    } else {
        // ---- consumers -----------------------------------------------------------------
        const float shift = CHECK ? a.shift[0] : 0.0f;
        const float dshift = CHECK ? a.shift[1] : 0.0f;
        ResAcc racc;                          // residual sums of this lane over its rows
        const int lx = warp * 32 + lane + kRowsHalo;
        const int x = x0 + lx - kRowsHalo;
        bool ok = true;
        for (int t = 0; t < nrows && ok; ++t) {
            ok = bar_wait_bounded(full + t % S, (unsigned)(t / S) & 1u);
            if (!ok || t < 2)
                continue;
            // output row y = y0 - 2 + t from input rows y - 1, y, y + 1
            const int y = y0 - 2 + t;
            const float *sm = ring + (size_t)((t - 2) % S) * slot_floats;
            const float *s0 = ring + (size_t)((t - 1) % S) * slot_floats;
            const float *sp = ring + (size_t)(t % S) * slot_floats;
            if (x < g.nx) {
                const int o = y * p + x;
                const float r0 = s0[8 * RW + lx];
                float f[8];
                if (interior(g, x, y)) {
                    f[0] = dev1(s0[0 * RW + lx - 1], wgt(1), s0[8 * RW + lx - 1], r0);
                    f[1] = dev1(sm[1 * RW + lx], wgt(2), sm[8 * RW + lx], r0);
                    f[2] = dev1(s0[2 * RW + lx + 1], wgt(3), s0[8 * RW + lx + 1], r0);
                    f[3] = dev1(sp[3 * RW + lx], wgt(4), sp[8 * RW + lx], r0);
                    f[4] = dev1(sm[4 * RW + lx - 1], wgt(5), sm[8 * RW + lx - 1], r0);
                    f[5] = dev1(sm[5 * RW + lx + 1], wgt(6), sm[8 * RW + lx + 1], r0);
                    f[6] = dev1(sp[6 * RW + lx + 1], wgt(7), sp[8 * RW + lx + 1], r0);
                    f[7] = dev1(sp[7 * RW + lx - 1], wgt(8), sp[8 * RW + lx - 1], r0);
                } else {
                    gather_a(a.fin, a.R, g, a.Pb, x, y, o, f);
                }
                const float dP = pressure_of(f);
                const float it = s0[9 * RW + lx];
                float F = a.Fp ? s0[10 * RW + lx] : 0.0f;
                for (int w = 0; w < a.w.n; ++w)
                    if (o == a.w.idx[w])
                        F += a.w.fp[w];
                const float Fq = 0.125f * F;   // w_bar_i = 1/8 (Eq. 3-5a)
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    a.fout[i][o] = collide1(f[i], wgt(i + 1), dP, it, Fq);
                if (CHECK)
                    racc.add((dP - a.Pio[o]) - dshift, (r0 - shift) + dP);
                if (WRITE_P)
                    a.Pio[o] = dP;
            }
            // row t - 2 is no longer needed by this warp
            __syncwarp();
            if (lane == 0)
                bar_arrive(empty + (t - 2) % S);
        }
        if (!ok) {
            // poison this warp's columns of the block's rows
            failed = 1;
            const float nan = __int_as_float(0x7fc00000);
            if (x < g.nx)
                for (int y = y0; y < y1; ++y)
                    for (int i = 0; i < 8; ++i)
                        a.fout[i][y * p + x] = nan;
        }
        if (CHECK) {
            double v[4];
            racc.warp_totals(v);
            if (lane == 0) {
                red[warp][0] = v[0];
                red[warp][1] = v[1];
                red[warp][2] = v[2];
                red[warp][3] = v[3];
            }
        }
    }
    __syncthreads();
    if (CHECK && threadIdx.x < 4) {
        double sum = 0.0;
        for (int w = 0; w < CW; ++w)
            sum += red[w][threadIdx.x];
        a.partials[4 * blockIdx.x + threadIdx.x] = failed ? (double)__int_as_float(0x7fc00000) : sum;
    }
}

// ---------------------------------------------------------------------------------------
// Two sweeps per launch on staged rows (walls on every side; no periodic side).
//
// The producer stages input rows exactly as above.  Consumer warp w owns the 30 output
// columns [x0 + 30 w, x0 + 30 w + 30) of a strip of W = 30 CW columns; its 32 lanes compute
// the first sweep on those columns plus one on each side (the halo the second sweep pulls
// from), row after row, and lanes 1..30 compute the second sweep one row behind, writing the
// populations to global memory.  Each lane keeps its column's first-sweep values of the
// last rows in registers (all eight of the previous row, the three pulled from below of the
// row before); a pull from a neighbouring column takes the neighbour lane's value by a warp
// shuffle, so the two sweeps exchange nothing through shared memory.  Input row t
// (y = y0 - 2 + t) feeds the first sweep at rows y - 1 .. y + 1; a warp releases it after the
// first sweep at row y + 1.  The second sweep at row y takes R, 1/tau_f and w_bar F~_p of its
// node from the lane's registers and R of the neighbouring columns by shuffles.
// A node on a wall applies the wall rules of Sec. 4 to its own first-sweep values.  Both
// sweeps use the per-node arithmetic of the single sweep, so the result equals two single
// sweeps bit for bit.  CHECK: the residual sums of the second sweep against the first
// (no increment plane).  Waits are bounded as in k_pressure_rows; a warp that gives up
// poisons its columns with NaN.
// ---------------------------------------------------------------------------------------
// R around the node, rows y - 1 (m), y (c), y + 1 (p) and columns x - 1 (0), x (1), x + 1 (2)
struct RNbhd {
    float m0, m1, m2, c0, c1, c2, p0, p1, p2;
    __device__ __forceinline__ float at(int ex, int ey) const
    {
        // the source x - c_i of a pull: column offset -ex, row offset -ey
        if (ey == 1)
            return ex == 1 ? m0 : (ex == -1 ? m2 : m1);
        if (ey == -1)
            return ex == 1 ? p0 : (ex == -1 ? p2 : p1);
        return ex == 1 ? c0 : (ex == -1 ? c2 : c1);
    }
};

// a_I of the second sweep at a wall node: the first sweep's value nb of the neighbour
// x - c_I (already fetched from that neighbour's lane), or the wall rule of Sec. 4 on the
// node's own first-sweep value own_opp of direction opp(I)
template <int I>
__device__ __forceinline__ float second_pull(float nb, float own_opp, const RNbhd &R,
                                             const Geom &g, const float *const *Pb, int x, int y,
                                             float r0)
{
    constexpr int ex = cx(I), ey = cy(I);
    int side = -1;
    if (x - ex < 0 || x - ex >= g.nx)
        side = x - ex < 0 ? 0 : 1;
    else if (y - ey < 0 || y - ey >= g.ny)
        side = y - ey < 0 ? 2 : 3;
    if (side < 0)
        return dev1(nb, wgt(I), R.at(ex, ey), r0);
    const float b = own_opp;
    if (g.bc[side] == BC_NOFLUX)
        return b;
    const int k = side < 2 ? 2 * y + 1 - ey : 2 * x + 1 - ex;
    return -b + 2.0f * wgt(I) * (Pb[side][k] - r0);
}

// Consumer warp of k_pressure_rows2 in a block whose first-sweep footprint (columns
// x0 - 1 .. x0 + W, rows y0 - 1 .. y0 + H) holds no wall node and no well, so that every
// pull of both sweeps comes from a lattice neighbour.  It runs the general consumer's
// protocol (the same waits, releases and give-up rule) and the same per-node arithmetic, so
// it writes the same populations bit for bit, without the wall and well tests.  The row loop
// is unrolled by two: the values a row hands to the rows after it are kept in two register
// sets indexed by the row's parity, so none is copied from row to row.
//   one row later:  v_1, v_3 (directions 1, 3), 1/tau_f, w_bar F~_p, dP of the first sweep;
//   two rows later: v_2, v_5, v_6 (directions pulled from below) and R.
template <bool CHECK, bool HAS_FP, int CW, int S>
struct Rows2Interior {
    static constexpr int RW = 30 * CW + 2 * kRowsHalo;
    const PressureArgs &a;
    const float *ring;
    int slot_floats;
    uint64_t *full, *empty;
    int lane, lx, q;
    unsigned ph;
    const float *sm, *s0, *sp;     // staged input rows t - 2, t - 1, t
    int qm;                        // slot of row t - 2 (released after the first sweep)
    int o;                         // output offset of the second sweep's node
    bool owner, ok;
    float c0[2], c2[2], d1[2], d4[2], d5[2], rr[2], tt[2], qq[2], dd[2];
    ResAcc racc;
    float shift, dshift;

    __device__ __forceinline__ Rows2Interior(const PressureArgs &a_, const float *ring_, int sf,
                                             uint64_t *full_, uint64_t *empty_, int lane_,
                                             int lx_, int o0, bool owner_, float shift_,
                                             float dshift_)
        : a(a_), ring(ring_), slot_floats(sf), full(full_), empty(empty_), lane(lane_), lx(lx_),
          q(0), ph(0u), sm(ring_), s0(ring_), sp(ring_), qm(0), o(o0), owner(owner_), ok(true),
          shift(shift_), dshift(dshift_)
    {
    }

    // wait for input row t (the next one) and make (sm, s0, sp) rows t - 2, t - 1, t
    __device__ __forceinline__ bool next_row()
    {
        ok = bar_wait_bounded(full + q, ph);
        sm = s0;
        s0 = sp;
        sp = ring + (size_t)q * slot_floats;
        qm = q == 0 ? S - 2 : (q == 1 ? S - 1 : q - 2);
        if (++q == S) {
            q = 0;
            ph ^= 1u;
        }
        return ok;
    }

    // first sweep at the row of s0 from the staged rows (sm, s0, sp); then row t - 2 is
    // released
    __device__ __forceinline__ void first(float (&v)[8], float &r0, float &it, float &Fq,
                                          float &dP)
    {
        r0 = s0[8 * RW + lx];
        float f[8];
        f[0] = dev1(s0[0 * RW + lx - 1], wgt(1), s0[8 * RW + lx - 1], r0);
        f[1] = dev1(sm[1 * RW + lx], wgt(2), sm[8 * RW + lx], r0);
        f[2] = dev1(s0[2 * RW + lx + 1], wgt(3), s0[8 * RW + lx + 1], r0);
        f[3] = dev1(sp[3 * RW + lx], wgt(4), sp[8 * RW + lx], r0);
        f[4] = dev1(sm[4 * RW + lx - 1], wgt(5), sm[8 * RW + lx - 1], r0);
        f[5] = dev1(sm[5 * RW + lx + 1], wgt(6), sm[8 * RW + lx + 1], r0);
        f[6] = dev1(sp[6 * RW + lx + 1], wgt(7), sp[8 * RW + lx + 1], r0);
        f[7] = dev1(sp[7 * RW + lx - 1], wgt(8), sp[8 * RW + lx - 1], r0);
        dP = pressure_of(f);
        it = s0[9 * RW + lx];
        const float F = HAS_FP ? s0[10 * RW + lx] : 0.0f;
        Fq = 0.125f * F;   // w_bar_i = 1/8 (Eq. 3-5a)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v[i] = collide1(f[i], wgt(i + 1), dP, it, Fq);
        __syncwarp();
        if (lane == 0)
            bar_arrive(empty + qm);
    }

    template <int P>
    __device__ __forceinline__ void keep(const float (&v)[8], float r0, float it, float Fq,
                                         float dP)
    {
        c0[P] = v[0];
        c2[P] = v[2];
        d1[P] = v[1];
        d4[P] = v[4];
        d5[P] = v[5];
        rr[P] = r0;
        tt[P] = it;
        if (HAS_FP)
            qq[P] = Fq;
        if (CHECK)
            dd[P] = dP;
    }

    // a row whose first sweep has parity P (rows t >= 4): first sweep, then the second sweep
    // one row behind it, from the register sets of both parities and warp shuffles
    template <int P>
    __device__ __forceinline__ void both()
    {
        float v[8], r0, it, Fq, dP1;
        first(v, r0, it, Fq, dP1);
        const float Rm = rr[P], Rc = rr[1 - P];
        const float m0 = __shfl_up_sync(0xffffffffu, Rm, 1);
        const float c0r = __shfl_up_sync(0xffffffffu, Rc, 1);
        const float p0 = __shfl_up_sync(0xffffffffu, r0, 1);
        const float m2 = __shfl_down_sync(0xffffffffu, Rm, 1);
        const float c2r = __shfl_down_sync(0xffffffffu, Rc, 1);
        const float p2 = __shfl_down_sync(0xffffffffu, r0, 1);
        float f[8];
        f[0] = dev1(__shfl_up_sync(0xffffffffu, c0[1 - P], 1), wgt(1), c0r, Rc);
        f[1] = dev1(d1[P], wgt(2), Rm, Rc);
        f[2] = dev1(__shfl_down_sync(0xffffffffu, c2[1 - P], 1), wgt(3), c2r, Rc);
        f[3] = dev1(v[3], wgt(4), r0, Rc);
        f[4] = dev1(__shfl_up_sync(0xffffffffu, d4[P], 1), wgt(5), m0, Rc);
        f[5] = dev1(__shfl_down_sync(0xffffffffu, d5[P], 1), wgt(6), m2, Rc);
        f[6] = dev1(__shfl_down_sync(0xffffffffu, v[6], 1), wgt(7), p2, Rc);
        f[7] = dev1(__shfl_up_sync(0xffffffffu, v[7], 1), wgt(8), p0, Rc);
        const float dP = pressure_of(f);
        if (owner) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a.fout[i][o] = collide1(f[i], wgt(i + 1), dP, tt[1 - P], HAS_FP ? qq[1 - P] : 0.0f);
            if (CHECK)
                racc.add((dP - dd[1 - P]) - dshift, (Rc - shift) + dP);
        }
        o += a.g.pitch;
        keep<P>(v, r0, it, Fq, dP1);
    }

    // rows 0 .. nrows - 1 of the block; false when a wait gave up
    __device__ __forceinline__ bool run(int nrows)
    {
        if (!next_row() || !next_row())
            return false;
        float v[8], r0, it, Fq, dP;
        if (!next_row())
            return false;
        first(v, r0, it, Fq, dP);
        keep<0>(v, r0, it, Fq, dP);
        if (!next_row())
            return false;
        first(v, r0, it, Fq, dP);
        keep<1>(v, r0, it, Fq, dP);
        int t = 4;
        for (; t + 1 < nrows; t += 2) {
            if (!next_row())
                return false;
            both<0>();
            if (!next_row())
                return false;
            both<1>();
        }
        if (t < nrows) {
            if (!next_row())
                return false;
            both<0>();
        }
        return true;
    }
};

template <bool CHECK, int CW, int S, int MINB>
__global__ void __launch_bounds__(32 * (CW + 1), MINB) k_pressure_rows2(const __grid_constant__ PressureArgs a,
                                                                  int H)
{
    constexpr int W = 30 * CW;
    constexpr int RW = W + 2 * kRowsHalo;          // floats per staged plane row
    const int npl = a.Fp ? 11 : 10;
    const int slot_floats = npl * RW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + S;
    float *ring = reinterpret_cast<float *>(smem + kRowsBarBytes);
    __shared__ double red[CW][4];
    __shared__ int failed;
    const Geom &g = a.g;
    const int p = g.pitch;
    const int strips = (g.nx + W - 1) / W;
    const int x0 = (blockIdx.x % strips) * W;
    const int y0 = (blockIdx.x / strips) * H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (y0 >= g.ny) {                              // not produced by rows_grid; kept safe
        if (CHECK && threadIdx.x < 4)
            a.partials[4 * blockIdx.x + threadIdx.x] = 0.0;
        return;
    }
    const int y1 = y0 + H < g.ny ? y0 + H : g.ny;
    const int nrows = y1 - y0 + 4;                 // input rows y0 - 2 .. y1 + 1
    const int xa = x0 - kRowsHalo > 0 ? x0 - kRowsHalo : 0;
    const int xb = x0 + W + kRowsHalo < p ? x0 + W + kRowsHalo : p;
    const unsigned seg = (unsigned)(xb - xa) * 4u;
    const int soff = xa - (x0 - kRowsHalo);
    // no wall node and no well among the first sweep's nodes x0 - 1 .. x0 + W,
    // y0 - 1 .. y1 (the second sweep's nodes lie inside them)
    bool interior_block = x0 >= 2 && x0 + W <= g.nx - 2 && y0 >= 2 && y1 <= g.ny - 2;
    for (int w = 0; w < a.w.n && interior_block; ++w) {
        const int wy = a.w.idx[w] / p, wx = a.w.idx[w] - wy * p;
        if (wx >= x0 - 1 && wx <= x0 + W && wy >= y0 - 1 && wy <= y1)
            interior_block = false;
    }

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            bar_init(full + q, 1);
            bar_init(empty + q, CW);
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == CW) {
        // ---- producer ------------------------------------------------------------------
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nrows; ++t) {
                const int q = t % S;
                if (t >= S && !bar_wait_bounded(empty + q, (unsigned)(t / S - 1) & 1u)) {
                    failed = 1;
                    break;
                }
                // the first row feeds only the c_y = +1 pulls of the first sweep's top row,
                // the last only the c_y = -1 pulls of its bottom row; both also give R
                const int r = y0 - 2 + t;
                unsigned m = npl == 11 ? 0x7FFu : 0x3FFu;
                if (r < 0 || r >= g.ny)
                    m = 0u;
                else if (t == 0)
                    m = (1u << 1) | (1u << 4) | (1u << 5) | (1u << 8);
                else if (t == nrows - 1)
                    m = (1u << 3) | (1u << 6) | (1u << 7) | (1u << 8);
                if (!m) {
                    bar_arrive(full + q);
                } else {
                    bar_arrive_tx(full + q, (unsigned)__popc(m) * seg);
                    const size_t roff = (size_t)r * p + xa;
                    float *slot = ring + (size_t)q * slot_floats + soff;
#pragma unroll
                    for (int pl = 0; pl < kRowsMaxPlanes; ++pl) {
                        if (!(m & (1u << pl)))
                            continue;
                        const float *src = pl < 8 ? a.fin[pl]
                                                  : (pl == 8 ? a.R : (pl == 9 ? a.inv_tau : a.Fp));
                        bulk_g2s(slot + pl * RW, src + roff, seg, full + q);
                    }
                }
                issued = t + 1;
            }
            for (int t = issued - S > 0 ? issued - S : 0; t < issued; ++t)
                bar_wait_bounded(full + t % S, (unsigned)(t / S) & 1u);
        }
    } else if (interior_block) {
        // ---- consumers of a block without walls or wells -------------------------------
        const int x = x0 - 1 + 30 * warp + lane;
        const bool owner = lane >= 1 && lane <= 30;
        bool done;
        ResAcc racc;
        if (a.Fp) {
            Rows2Interior<CHECK, true, CW, S> c(a, ring, slot_floats, full, empty, lane,
                                                x - (x0 - kRowsHalo), y0 * p + x, owner,
                                                CHECK ? a.shift[0] : 0.0f,
                                                CHECK ? a.shift[1] : 0.0f);
            done = c.run(nrows);
            racc = c.racc;
        } else {
            Rows2Interior<CHECK, false, CW, S> c(a, ring, slot_floats, full, empty, lane,
                                                 x - (x0 - kRowsHalo), y0 * p + x, owner,
                                                 CHECK ? a.shift[0] : 0.0f,
                                                 CHECK ? a.shift[1] : 0.0f);
            done = c.run(nrows);
            racc = c.racc;
        }
        if (!done) {
            failed = 1;
            const float nan = __int_as_float(0x7fc00000);
            if (owner)
                for (int y = y0; y < y1; ++y)
                    for (int i = 0; i < 8; ++i)
                        a.fout[i][y * p + x] = nan;
        }
        if (CHECK) {
            double v[4];
            racc.warp_totals(v);
            if (lane == 0) {
                red[warp][0] = v[0];
                red[warp][1] = v[1];
                red[warp][2] = v[2];
                red[warp][3] = v[3];
            }
        }
    } else {
        // ---- consumers -----------------------------------------------------------------
        const float shift = CHECK ? a.shift[0] : 0.0f;
        const float dshift = CHECK ? a.shift[1] : 0.0f;
        ResAcc racc;
        const int x = x0 - 1 + 30 * warp + lane;    // this lane's column (both sweeps)
        const int lx = x - (x0 - kRowsHalo);        // its column in a staged row
        const bool xin = x >= 0 && x < g.nx;
        const bool owner = lane >= 1 && lane <= 30 && x < g.nx;
        // this lane's R, 1/tau_f, w_bar F~_p and first-sweep dP of its last three first-sweep
        // rows (a: two arrivals ago, b: one, c: this one): the second sweep reads them from
        // registers and its neighbours' by shuffles, so a staged row is released as soon as
        // the first sweep is done with it
        float ra = 0.0f, rb = 0.0f, rc = 0.0f, tb = 0.0f, tc = 0.0f, qb = 0.0f, qc = 0.0f;
        float db = 0.0f, dc = 0.0f;
        // first-sweep populations of this lane's column: v = the newest row, h1 = the one
        // before (all planes: the wall rules read the node's own values), h2 = the one before
        // that (only the planes pulled from the row below: directions 2, 5, 6)
        float v[8], h1[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v[i] = h1[i] = 0.0f;
        float h2_1 = 0.0f, h2_4 = 0.0f, h2_5 = 0.0f;
        // wells in this lane's column (the source test runs only there)
        bool wcol = false;
        for (int w = 0; w < a.w.n; ++w)
            wcol = wcol || (xin && a.w.idx[w] % p == x);
        const bool xinner = x > 0 && x < g.nx - 1;
        // slots and parity advance by increments (no division in the row loop): input rows
        // t - 2, t - 1, t in slots qm, q0, qp
        int q = 0, qm = 0, q0 = 0;
        unsigned ph = 0u;
        bool ok = true;
        for (int t = 0; t < nrows && ok; ++t) {
            ok = bar_wait_bounded(full + q, ph);
            const int qp = q;
            if (++q == S) {
                q = 0;
                ph ^= 1u;
            }
            if (!ok)
                break;
            if (t < 2) {
                qm = q0;
                q0 = qp;
                continue;
            }
            // first sweep at row ys from input rows ys - 1, ys, ys + 1 (arrivals t-2..t)
            const int ys = y0 - 3 + t;
            {
                const float *sm = ring + (size_t)qm * slot_floats;
                const float *s0 = ring + (size_t)q0 * slot_floats;
                const float *sp = ring + (size_t)qp * slot_floats;
                h2_1 = h1[1];
                h2_4 = h1[4];
                h2_5 = h1[5];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    h1[i] = v[i];
                    v[i] = 0.0f;
                }
                ra = rb;
                rb = rc;
                tb = tc;
                qb = qc;
                db = dc;
                rc = tc = qc = dc = 0.0f;
                if (xin && ys >= 0 && ys < g.ny) {
                    const int o = ys * p + x;
                    const float r0 = s0[8 * RW + lx];
                    float f[8];
                    if (xinner && ys > 0 && ys < g.ny - 1) {
                        f[0] = dev1(s0[0 * RW + lx - 1], wgt(1), s0[8 * RW + lx - 1], r0);
                        f[1] = dev1(sm[1 * RW + lx], wgt(2), sm[8 * RW + lx], r0);
                        f[2] = dev1(s0[2 * RW + lx + 1], wgt(3), s0[8 * RW + lx + 1], r0);
                        f[3] = dev1(sp[3 * RW + lx], wgt(4), sp[8 * RW + lx], r0);
                        f[4] = dev1(sm[4 * RW + lx - 1], wgt(5), sm[8 * RW + lx - 1], r0);
                        f[5] = dev1(sm[5 * RW + lx + 1], wgt(6), sm[8 * RW + lx + 1], r0);
                        f[6] = dev1(sp[6 * RW + lx + 1], wgt(7), sp[8 * RW + lx + 1], r0);
                        f[7] = dev1(sp[7 * RW + lx - 1], wgt(8), sp[8 * RW + lx - 1], r0);
                    } else {
                        gather_a(a.fin, a.R, g, a.Pb, x, ys, o, f);
                    }
                    const float dP = pressure_of(f);
                    const float it = s0[9 * RW + lx];
                    float F = a.Fp ? s0[10 * RW + lx] : 0.0f;
                    if (wcol)
                        for (int w = 0; w < a.w.n; ++w)
                            if (o == a.w.idx[w])
                                F += a.w.fp[w];
                    const float Fq = 0.125f * F;   // w_bar_i = 1/8 (Eq. 3-5a)
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        v[i] = collide1(f[i], wgt(i + 1), dP, it, Fq);
                    rc = r0;
                    tc = it;
                    qc = Fq;
                    dc = dP;
                }
                __syncwarp();
                // input row t - 2 is no longer needed by this warp
                if (lane == 0)
                    bar_arrive(empty + qm);
                qm = q0;
                q0 = qp;
            }
            if (t < 4)
                continue;
            // second sweep at row y2 = ys - 1 from the first sweep's rows y2 - 1, y2, y2 + 1:
            // the neighbour x - c_i of each pull sits in this lane or the next one over
            const int y2 = ys - 1;
            RNbhd Rn;
            Rn.m1 = ra;
            Rn.c1 = rb;
            Rn.p1 = rc;
            Rn.m0 = __shfl_up_sync(0xffffffffu, ra, 1);
            Rn.c0 = __shfl_up_sync(0xffffffffu, rb, 1);
            Rn.p0 = __shfl_up_sync(0xffffffffu, rc, 1);
            Rn.m2 = __shfl_down_sync(0xffffffffu, ra, 1);
            Rn.c2 = __shfl_down_sync(0xffffffffu, rb, 1);
            Rn.p2 = __shfl_down_sync(0xffffffffu, rc, 1);
            float nb[8];
            nb[0] = __shfl_up_sync(0xffffffffu, h1[0], 1);     // 1: from (x-1, y2)
            nb[1] = h2_1;                                      // 2: from (x, y2-1)
            nb[2] = __shfl_down_sync(0xffffffffu, h1[2], 1);   // 3: from (x+1, y2)
            nb[3] = v[3];                                      // 4: from (x, y2+1)
            nb[4] = __shfl_up_sync(0xffffffffu, h2_4, 1);      // 5: from (x-1, y2-1)
            nb[5] = __shfl_down_sync(0xffffffffu, h2_5, 1);    // 6: from (x+1, y2-1)
            nb[6] = __shfl_down_sync(0xffffffffu, v[6], 1);    // 7: from (x+1, y2+1)
            nb[7] = __shfl_up_sync(0xffffffffu, v[7], 1);      // 8: from (x-1, y2+1)
            if (owner && y2 < g.ny) {
                const float r0 = rb;
                float f[8];
                if (xinner && y2 > 0 && y2 < g.ny - 1) {
                    f[0] = dev1(nb[0], wgt(1), Rn.c0, r0);
                    f[1] = dev1(nb[1], wgt(2), Rn.m1, r0);
                    f[2] = dev1(nb[2], wgt(3), Rn.c2, r0);
                    f[3] = dev1(nb[3], wgt(4), Rn.p1, r0);
                    f[4] = dev1(nb[4], wgt(5), Rn.m0, r0);
                    f[5] = dev1(nb[5], wgt(6), Rn.m2, r0);
                    f[6] = dev1(nb[6], wgt(7), Rn.p2, r0);
                    f[7] = dev1(nb[7], wgt(8), Rn.p0, r0);
                } else {
                    f[0] = second_pull<1>(nb[0], h1[opp(1) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[1] = second_pull<2>(nb[1], h1[opp(2) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[2] = second_pull<3>(nb[2], h1[opp(3) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[3] = second_pull<4>(nb[3], h1[opp(4) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[4] = second_pull<5>(nb[4], h1[opp(5) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[5] = second_pull<6>(nb[5], h1[opp(6) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[6] = second_pull<7>(nb[6], h1[opp(7) - 1], Rn, g, a.Pb, x, y2, r0);
                    f[7] = second_pull<8>(nb[7], h1[opp(8) - 1], Rn, g, a.Pb, x, y2, r0);
                }
                const int o = y2 * p + x;
                const float dP = pressure_of(f);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    a.fout[i][o] = collide1(f[i], wgt(i + 1), dP, tb, qb);
                if (CHECK)
                    racc.add((dP - db) - dshift, (r0 - shift) + dP);
            }
        }
        if (!ok) {
            failed = 1;
            const float nan = __int_as_float(0x7fc00000);
            if (owner)
                for (int y = y0; y < y1; ++y)
                    for (int i = 0; i < 8; ++i)
                        a.fout[i][y * p + x] = nan;
        }
        if (CHECK) {
            double v[4];
            racc.warp_totals(v);
            if (lane == 0) {
                red[warp][0] = v[0];
                red[warp][1] = v[1];
                red[warp][2] = v[2];
                red[warp][3] = v[3];
            }
        }
    }
    __syncthreads();
    if (CHECK && threadIdx.x < 4) {
        double sum = 0.0;
        for (int w = 0; w < CW; ++w)
            sum += red[w][threadIdx.x];
        a.partials[4 * blockIdx.x + threadIdx.x] = failed ? (double)__int_as_float(0x7fc00000) : sum;
    }
}

// ---------------------------------------------------------------------------------------
// Two sweeps per launch with the inputs read straight from global memory (lattices with walls
// on every side).  The consumer logic of k_pressure_rows2 without the staging: warp w of a
// block owns 30 columns, walks the block's H rows, computes the first sweep on its 32
// columns with the scalar gather (L1/L2 hits where the lattice stays in L2) and the second
// sweep one row behind from register history and shuffles.  No producer, no mbarrier, no
// shared memory but the block's residual reduction: meant for lattices small enough that
// their populations stay in L2 between sweeps, where the staged pipeline's per-row latency
// dominates.  Same per-node arithmetic, so results equal two single sweeps bit for bit.
// The register history and the second sweep are written out here as in k_pressure_rows2
// rather than shared through a helper: the helper version compiled to different register
// counts (64 instead of 48 for the 8-warp plain launch, 72 instead of 64 for the 4-warp
// checking one), and these counts set the blocks resident per SM.
// ---------------------------------------------------------------------------------------
// Block bidx of the lattice of `a` (strips of W = 30 CW columns by H rows); CHECK: the block's
// four residual sums go to part[0 .. 3].  Every thread of the block calls it.
template <bool CHECK, int CW>
__device__ __forceinline__ void pair_direct_block(const PressureArgs &a, int H, int bidx,
                                                  double *part)
{
    constexpr int W = 30 * CW;
    __shared__ double red[CW][4];
    const Geom &g = a.g;
    const int p = g.pitch;
    const int strips = (g.nx + W - 1) / W;
    const int x0 = (bidx % strips) * W;
    const int y0 = (bidx / strips) * H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float shift = CHECK ? a.shift[0] : 0.0f;
    const float dshift = CHECK ? a.shift[1] : 0.0f;
    ResAcc racc;
    const int y1 = y0 + H < g.ny ? y0 + H : g.ny;
    const int x = x0 - 1 + 30 * warp + lane;
    const bool xin = x >= 0 && x < g.nx;
    const bool owner = lane >= 1 && lane <= 30 && x < g.nx;
    float ra = 0.0f, rb = 0.0f, rc = 0.0f, tb = 0.0f, tc = 0.0f, qb = 0.0f, qc = 0.0f;
    float db = 0.0f, dc = 0.0f;
    float v[8], h1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        v[i] = h1[i] = 0.0f;
    float h2_1 = 0.0f, h2_4 = 0.0f, h2_5 = 0.0f;
    // the first sweep runs on rows y0 - 1 .. y1 (one more on each side), the second one row
    // behind it on rows y0 .. y1 - 1
    for (int ys = y0 - 1; ys <= y1 && y0 < g.ny; ++ys) {
        h2_1 = h1[1];
        h2_4 = h1[4];
        h2_5 = h1[5];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            h1[i] = v[i];
            v[i] = 0.0f;
        }
        ra = rb;
        rb = rc;
        tb = tc;
        qb = qc;
        db = dc;
        rc = tc = qc = dc = 0.0f;
        if (xin && ys >= 0 && ys < g.ny) {
            const int o = ys * p + x;
            const float r0 = a.R[o];
            float f[8];
            gather_a(a.fin, a.R, g, a.Pb, x, ys, o, f);
            const float dP = pressure_of(f);
            const float it = a.inv_tau[o];
            float F = a.Fp ? a.Fp[o] : 0.0f;
            for (int w = 0; w < a.w.n; ++w)
                if (o == a.w.idx[w])
                    F += a.w.fp[w];
            const float Fq = 0.125f * F;   // w_bar_i = 1/8 (Eq. 3-5a)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                v[i] = collide1(f[i], wgt(i + 1), dP, it, Fq);
            rc = r0;
            tc = it;
            qc = Fq;
            dc = dP;
        }
        const int y2 = ys - 1;
        if (y2 < y0)
            continue;
        RNbhd Rn;
        Rn.m1 = ra;
        Rn.c1 = rb;
        Rn.p1 = rc;
        Rn.m0 = __shfl_up_sync(0xffffffffu, ra, 1);
        Rn.c0 = __shfl_up_sync(0xffffffffu, rb, 1);
        Rn.p0 = __shfl_up_sync(0xffffffffu, rc, 1);
        Rn.m2 = __shfl_down_sync(0xffffffffu, ra, 1);
        Rn.c2 = __shfl_down_sync(0xffffffffu, rb, 1);
        Rn.p2 = __shfl_down_sync(0xffffffffu, rc, 1);
        float nb[8];
        nb[0] = __shfl_up_sync(0xffffffffu, h1[0], 1);
        nb[1] = h2_1;
        nb[2] = __shfl_down_sync(0xffffffffu, h1[2], 1);
        nb[3] = v[3];
        nb[4] = __shfl_up_sync(0xffffffffu, h2_4, 1);
        nb[5] = __shfl_down_sync(0xffffffffu, h2_5, 1);
        nb[6] = __shfl_down_sync(0xffffffffu, v[6], 1);
        nb[7] = __shfl_up_sync(0xffffffffu, v[7], 1);
        if (owner && y2 < g.ny) {
            const float r0 = rb;
            float f[8];
            if (x > 0 && x < g.nx - 1 && y2 > 0 && y2 < g.ny - 1) {
                f[0] = dev1(nb[0], wgt(1), Rn.c0, r0);
                f[1] = dev1(nb[1], wgt(2), Rn.m1, r0);
                f[2] = dev1(nb[2], wgt(3), Rn.c2, r0);
                f[3] = dev1(nb[3], wgt(4), Rn.p1, r0);
                f[4] = dev1(nb[4], wgt(5), Rn.m0, r0);
                f[5] = dev1(nb[5], wgt(6), Rn.m2, r0);
                f[6] = dev1(nb[6], wgt(7), Rn.p2, r0);
                f[7] = dev1(nb[7], wgt(8), Rn.p0, r0);
            } else {
                f[0] = second_pull<1>(nb[0], h1[opp(1) - 1], Rn, g, a.Pb, x, y2, r0);
                f[1] = second_pull<2>(nb[1], h1[opp(2) - 1], Rn, g, a.Pb, x, y2, r0);
                f[2] = second_pull<3>(nb[2], h1[opp(3) - 1], Rn, g, a.Pb, x, y2, r0);
                f[3] = second_pull<4>(nb[3], h1[opp(4) - 1], Rn, g, a.Pb, x, y2, r0);
                f[4] = second_pull<5>(nb[4], h1[opp(5) - 1], Rn, g, a.Pb, x, y2, r0);
                f[5] = second_pull<6>(nb[5], h1[opp(6) - 1], Rn, g, a.Pb, x, y2, r0);
                f[6] = second_pull<7>(nb[6], h1[opp(7) - 1], Rn, g, a.Pb, x, y2, r0);
                f[7] = second_pull<8>(nb[7], h1[opp(8) - 1], Rn, g, a.Pb, x, y2, r0);
            }
            const int o = y2 * p + x;
            const float dP = pressure_of(f);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a.fout[i][o] = collide1(f[i], wgt(i + 1), dP, tb, qb);
            if (CHECK)
                racc.add((dP - db) - dshift, (r0 - shift) + dP);
        }
    }
    if (CHECK) {
        double vsum[4];
        racc.warp_totals(vsum);
        if (lane == 0)
            for (int c = 0; c < 4; ++c)
                red[warp][c] = vsum[c];
        __syncthreads();
        if (threadIdx.x < 4) {
            double sum = 0.0;
            for (int w = 0; w < CW; ++w)
                sum += red[w][threadIdx.x];
            part[threadIdx.x] = sum;
        }
    }
}

template <bool CHECK, int CW>
__global__ void __launch_bounds__(32 * CW) k_pressure_pair_direct(const __grid_constant__ PressureArgs a,
                                                                 int H)
{
    pair_direct_block<CHECK, CW>(a, H, blockIdx.x, CHECK ? a.partials + 4 * blockIdx.x : nullptr);
}

// Two sweeps with direct loads over several lattices in one launch (the batch's members of
// 512^2 nodes and more): item t = (member m, block b) runs block b of member m's lattice with
// the argument block pa[2 m + parity] and H[m] rows per block; CHECK: its residual sums go to
// parts[4 (pb0[m] + b) ..].  The list holds the blocks of the members still iterating.
template <bool CHECK>
__global__ void __launch_bounds__(128) k_pair_batch(const PressureArgs *__restrict__ pa,
                                                    const int *__restrict__ H,
                                                    const int *__restrict__ pb0,
                                                    const int2 *__restrict__ items,
                                                    const int *__restrict__ nitems, int parity,
                                                    double *__restrict__ parts)
{
    const int n = *nitems;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int2 e = items[t];
        pair_direct_block<CHECK, 4>(pa[2 * e.x + parity], H[e.x], e.y,
                                    CHECK ? parts + 4 * ((size_t)pb0[e.x] + e.y) : nullptr);
        if (CHECK)
            __syncthreads();                           // the reduction array is reused
    }
}

void *pair_direct_func(int cw, bool check)
{
    if (cw == 4)
        return check ? (void *)k_pressure_pair_direct<true, 4> : (void *)k_pressure_pair_direct<false, 4>;
    return check ? (void *)k_pressure_pair_direct<true, 8> : (void *)k_pressure_pair_direct<false, 8>;
}

// Register caps (blocks per SM the compiler must allow): six 4-warp blocks (64 registers) or
// three 8-warp ones; the dense variant's plain launch allows seven 4-warp blocks (56 registers,
// a few bytes spilled) while its checking launch keeps six (no spills).
template <int CW, int S, bool DENSE>
void *rows2_func_t(bool check)
{
    constexpr int base = CW == 4 ? 6 : 3;
    return check ? (void *)k_pressure_rows2<true, CW, S, base>
                 : (void *)k_pressure_rows2<false, CW, S, DENSE ? base + 1 : base>;
}

// the two-sweep shapes built: (consumer warps, ring slots [+ kRows2Dense])
void *rows2_func(int cw, int slots, bool check)
{
    if (cw == 4) {
        if (slots == 6 + lbm2p_launch::kRows2Dense)
            return rows2_func_t<4, 6, true>(check);
        return slots == 6 ? rows2_func_t<4, 6, false>(check) : rows2_func_t<4, 8, false>(check);
    }
    return slots == 4 ? rows2_func_t<8, 4, false>(check) : rows2_func_t<8, 6, false>(check);
}

template <int CW, int S>
void *rows_func_t(bool check, bool write_p)
{
    return check ? (write_p ? (void *)k_pressure_rows<true, true, CW, S>
                            : (void *)k_pressure_rows<true, false, CW, S>)
                 : (write_p ? (void *)k_pressure_rows<false, true, CW, S>
                            : (void *)k_pressure_rows<false, false, CW, S>);
}

// the shapes built: (strip width, ring slots)
void *rows_func(int width, int slots, bool check, bool write_p)
{
    if (width == 128)
        return rows_func_t<4, 8>(check, write_p);
    return slots == 6 ? rows_func_t<8, 6>(check, write_p) : rows_func_t<8, 8>(check, write_p);
}

}  // namespace
}  // namespace lbm2p_dev

namespace lbm2p_launch {

using lbm2p_dev::PressureArgs;

bool rows_shape_ok(int width, int slots)
{
    return (width == 128 && slots == 8) || (width == 256 && (slots == 6 || slots == 8));
}

int rows_threads(int width)
{
    return width + 32;
}

size_t rows_smem_bytes(int width, int slots, bool has_fp)
{
    const size_t rw = (size_t)width + 2 * lbm2p_dev::kRowsHalo;
    return 128 + lbm2p_dev::kRowsBarBytes + (size_t)slots * (has_fp ? 11 : 10) * rw * sizeof(float);
}

long long rows_grid(int width, int H, int nx, int ny)
{
    return (long long)((nx + width - 1) / width) * ((ny + H - 1) / H);
}

cudaError_t rows_prepare(int width, int slots)
{
    const int bytes = (int)rows_smem_bytes(width, slots, true);
    for (bool c : {false, true})
        for (bool w : {false, true}) {
            cudaError_t e = cudaFuncSetAttribute(lbm2p_dev::rows_func(width, slots, c, w),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess)
                return e;
        }
    return cudaSuccess;
}

int rows_blocks_per_sm(int width, int slots, bool has_fp)
{
    int lo = 1 << 30;
    for (bool c : {false, true})
        for (bool w : {false, true}) {
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b, lbm2p_dev::rows_func(width, slots, c, w), rows_threads(width),
                rows_smem_bytes(width, slots, has_fp));
            lo = b < lo ? b : lo;
        }
    return lo;
}

void pressure_sweep_rows(const PressureArgs &a, bool check, bool write_p, int width, int slots,
                         int H, int grid, void *stream)
{
    void *args[] = {(void *)&a, (void *)&H};
    cudaLaunchKernel(lbm2p_dev::rows_func(width, slots, check, write_p), dim3(grid),
                     dim3(rows_threads(width)), args, rows_smem_bytes(width, slots, a.Fp != nullptr),
                     reinterpret_cast<cudaStream_t>(stream));
}

cudaError_t node_pressure_rows(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                               const PressureArgs &a, bool check, bool write_p, int width,
                               int slots, int H, int grid)
{
    cudaKernelNodeParams prm{};
    prm.func = lbm2p_dev::rows_func(width, slots, check, write_p);
    prm.gridDim = dim3((unsigned)grid);
    prm.blockDim = dim3((unsigned)rows_threads(width));
    prm.sharedMemBytes = (unsigned)rows_smem_bytes(width, slots, a.Fp != nullptr);
    void *args[] = {(void *)&a, (void *)&H};
    prm.kernelParams = args;
    prm.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &prm);
}


// ---- two sweeps per launch on staged rows ----------------------------------------------
bool rows2_shape_ok(int cw, int slots)
{
    if (cw == 4 && slots == 6 + kRows2Dense)
        return true;
    return (cw == 4 && (slots == 6 || slots == 8)) || (cw == 8 && (slots == 4 || slots == 6));
}

int rows2_width(int cw)
{
    return 30 * cw;
}

size_t rows2_smem_bytes(int cw, int slots, bool has_fp)
{
    slots &= kRows2Dense - 1;
    const size_t rw = (size_t)rows2_width(cw) + 2 * lbm2p_dev::kRowsHalo;
    return 128 + lbm2p_dev::kRowsBarBytes + (size_t)slots * (has_fp ? 11 : 10) * rw * sizeof(float);
}

long long rows2_grid(int cw, int H, int nx, int ny)
{
    const int w = rows2_width(cw);
    return (long long)((nx + w - 1) / w) * ((ny + H - 1) / H);
}

cudaError_t rows2_prepare(int cw, int slots)
{
    const int bytes = (int)rows2_smem_bytes(cw, slots, true);
    for (bool c : {false, true}) {
        cudaError_t e = cudaFuncSetAttribute(lbm2p_dev::rows2_func(cw, slots, c),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

int rows2_blocks_per_sm(int cw, int slots, bool has_fp)
{
    int lo = 1 << 30;
    for (bool c : {false, true}) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lbm2p_dev::rows2_func(cw, slots, c),
                                                      32 * (cw + 1), rows2_smem_bytes(cw, slots, has_fp));
        lo = b < lo ? b : lo;
    }
    return lo;
}

void pressure_sweeps_rows2(const PressureArgs &a, bool check, int cw, int slots, int H, int grid,
                           void *stream)
{
    void *args[] = {(void *)&a, (void *)&H};
    cudaLaunchKernel(lbm2p_dev::rows2_func(cw, slots, check), dim3(grid), dim3(32 * (cw + 1)), args,
                     rows2_smem_bytes(cw, slots, a.Fp != nullptr),
                     reinterpret_cast<cudaStream_t>(stream));
}

cudaError_t node_pressure_rows2(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                                const PressureArgs &a, bool check, int cw, int slots, int H,
                                int grid)
{
    cudaKernelNodeParams prm{};
    prm.func = lbm2p_dev::rows2_func(cw, slots, check);
    prm.gridDim = dim3((unsigned)grid);
    prm.blockDim = dim3((unsigned)(32 * (cw + 1)));
    prm.sharedMemBytes = (unsigned)rows2_smem_bytes(cw, slots, a.Fp != nullptr);
    void *args[] = {(void *)&a, (void *)&H};
    prm.kernelParams = args;
    prm.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &prm);
}


// ---- two sweeps per launch with direct loads ------------------------------------------------
long long pair_direct_grid(int cw, int H, int nx, int ny)
{
    const int w = 30 * cw;
    return (long long)((nx + w - 1) / w) * ((ny + H - 1) / H);
}


void pressure_sweeps_pair_direct(const PressureArgs &a, bool check, int cw, int H, int grid,
                                 void *stream)
{
    void *args[] = {(void *)&a, (void *)&H};
    cudaLaunchKernel(lbm2p_dev::pair_direct_func(cw, check), dim3(grid), dim3(32 * cw), args, 0,
                     reinterpret_cast<cudaStream_t>(stream));
}

cudaError_t node_pressure_pair_direct(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                                      const PressureArgs &a, bool check, int cw, int H, int grid)
{
    cudaKernelNodeParams prm{};
    prm.func = lbm2p_dev::pair_direct_func(cw, check);
    prm.gridDim = dim3((unsigned)grid);
    prm.blockDim = dim3((unsigned)(32 * cw));
    prm.sharedMemBytes = 0;
    void *args[] = {(void *)&a, (void *)&H};
    prm.kernelParams = args;
    prm.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &prm);
}

int pair_batch_blocks_per_sm()
{
    int b1 = 0, b2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, lbm2p_dev::k_pair_batch<false>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, lbm2p_dev::k_pair_batch<true>, 128, 0);
    const int b = b1 < b2 ? b1 : b2;
    return b > 0 ? b : 1;
}

cudaError_t node_pair_batch(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                            const PressureArgs *pa, const int *H, const int *pb0,
                            const int2 *items, const int *nitems, int parity, bool check,
                            double *parts, int grid)
{
    cudaKernelNodeParams prm{};
    prm.func = check ? (void *)lbm2p_dev::k_pair_batch<true> : (void *)lbm2p_dev::k_pair_batch<false>;
    prm.gridDim = dim3((unsigned)grid);
    prm.blockDim = dim3(128u);
    prm.sharedMemBytes = 0;
    void *args[] = {(void *)&pa, (void *)&H, (void *)&pb0, (void *)&items, (void *)&nitems,
                    (void *)&parity, (void *)&parts};
    prm.kernelParams = args;
    prm.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &prm);
}

}  // namespace lbm2p_launch
