// FP16 storage of the pressure populations inside a sub-iteration (storage FP16_DEV).
//
// Between physical steps the state lives in the FP32 planes (deviations n_i = f_i^+ - w_i R).
// A pressure solve narrows them to FP16, sweeps on FP16, and widens the result back:
//   narrow:  s = 2^k chosen on the device from max |n_i| (2^12 headroom below FP16's range),
//            h_i = fp16(s n_i), Rh = R;
//   sweep:   a_i = h_i(x - c_i)/s + w_i (Rh(x - c_i) - Rh(x))  (walls as in the FP32 sweep),
//            dP = (9/5) sum a_i (Eq. 3-9a relative to Rh), then the BGK collision
//            (Eq. 2-1b) rebased onto the node's new pressure Rh' = Rh + dP:
//            h_i' = fp16(s [(1 - 1/tau_f)(a_i - w_i dP) + F~_p/8]),
//            so the stored values are the post-collision non-equilibrium parts and every
//            sweep's increment dP = P^k - P^{k-1} feeds the residual directly;
//   widen:   n_i = h_i / s, R = Rh.
// Arithmetic is FP32, the residual partials FP64, as in the FP32 sweep.  Bytes per node and
// sweep: 8 x (2 + 2) populations + 4 + 4 (Rh in, out) + 4 (1/tau_f) = 44 B.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm2p_async.cuh"
#include "lbm2p_device.cuh"
#include "lbm2p_node.cuh"

namespace lbm2p_dev {
namespace {

__device__ __forceinline__ float ld_h(const __half *p, int i, float inv_s)
{
    return __half2float(p[i]) * inv_s;
}

// a_I pulled into an edge node from FP16 planes (the wall rules of Sec. 4, deviation form)
template <int I>
__device__ __forceinline__ float pull_edge_h(const __half *__restrict__ n_i,
                                             const __half *__restrict__ n_opp,
                                             const float *__restrict__ R, const Geom &g,
                                             const float *const *Pb, int x, int y, float r0,
                                             float inv_s)
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
        return dev1(ld_h(n_i, src, inv_s), wgt(I), R[src], r0);
    }
    const float b = ld_h(n_opp, y * g.pitch + x, inv_s);
    if (g.bc[side] == BC_NOFLUX)
        return b;
    const int k = side < 2 ? 2 * y + 1 - ey : 2 * x + 1 - ex;
    return -b + 2.0f * wgt(I) * (Pb[side][k] - r0);
}

__global__ void __launch_bounds__(kBlock) k_absmax(const __grid_constant__ HalfConvertArgs a)
{
    const Geom &g = a.g;
    float m = 0.0f;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx) {
            const int o = y * g.pitch + x;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                m = fmaxf(m, fabsf(a.n32[i][o]));
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned int *>(&a.scale[2]), __float_as_uint(m));
}

// scale[0] = s = 2^k with s max|n| in [2^11, 2^12) (2^16 when the state is all zero, as
// after f = f^eq(P0); the host rescales at the first check), scale[1] = 1/s; scale[2] (the
// max) is cleared for the next solve
__global__ void k_set_scale(float *scale)
{
    const float m = scale[2];
    float s = 65536.0f;
    if (m > 0.0f && isfinite(m)) {
        int e;
        frexpf(m, &e);                 // m = f 2^e, f in [0.5, 1)
        int k = 12 - e;
        k = k < -100 ? -100 : (k > 100 ? 100 : k);
        s = ldexpf(1.0f, k);
    }
    scale[0] = s;
    scale[1] = 1.0f / s;
    scale[2] = 0.0f;
}

__global__ void __launch_bounds__(kBlock) k_narrow(const __grid_constant__ HalfConvertArgs a)
{
    const Geom &g = a.g;
    const float s = a.scale[0];
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx) {
            const int o = y * g.pitch + x;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a.n16[i][o] = __float2half_rn(a.n32[i][o] * s);
            a.Rh[o] = a.R[o];
        }
    }
}

// multiply every stored value by a power of two (exact within FP16's range)
__global__ void __launch_bounds__(kBlock) k_rescale(const __grid_constant__ HalfConvertArgs a,
                                                    float factor)
{
    const Geom &g = a.g;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx) {
            const int o = y * g.pitch + x;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a.n16[i][o] = __float2half_rn(__half2float(a.n16[i][o]) * factor);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_widen(const __grid_constant__ HalfConvertArgs a)
{
    const Geom &g = a.g;
    const float inv_s = a.scale[1];
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        if (x < g.nx) {
            const int o = y * g.pitch + x;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a.n32w[i][o] = __half2float(a.n16[i][o]) * inv_s;
            a.Rw[o] = a.Rh[o];
        }
    }
}

template <bool CHECK>
__global__ void __launch_bounds__(kBlock) k_pressure_h(const __grid_constant__ HalfSweepArgs a)
{
    const Geom &g = a.g;
    const int lane = threadIdx.x & 31;
    const float s = a.scale[0], inv_s = a.scale[1];
    ResAcc racc;                                  // residual sums of this thread
    float nmax = 0.0f;
    const float shift = CHECK ? a.shift[0] : 0.0f;
    const float dshift = CHECK ? a.shift[1] : 0.0f;
    const int p = g.pitch;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const int y = t / g.tiles_x;
        const int x = (t - y * g.tiles_x) * kBlock + threadIdx.x;
        float d = 0.0f, q = 0.0f;
        if (x < g.nx) {
            const int o = y * p + x;
            const float r0 = a.Rin[o];
            float f[8];
            if (interior(g, x, y)) {
                f[0] = dev1(ld_h(a.nin[0], o - 1, inv_s), wgt(1), a.Rin[o - 1], r0);
                f[1] = dev1(ld_h(a.nin[1], o - p, inv_s), wgt(2), a.Rin[o - p], r0);
                f[2] = dev1(ld_h(a.nin[2], o + 1, inv_s), wgt(3), a.Rin[o + 1], r0);
                f[3] = dev1(ld_h(a.nin[3], o + p, inv_s), wgt(4), a.Rin[o + p], r0);
                f[4] = dev1(ld_h(a.nin[4], o - p - 1, inv_s), wgt(5), a.Rin[o - p - 1], r0);
                f[5] = dev1(ld_h(a.nin[5], o - p + 1, inv_s), wgt(6), a.Rin[o - p + 1], r0);
                f[6] = dev1(ld_h(a.nin[6], o + p + 1, inv_s), wgt(7), a.Rin[o + p + 1], r0);
                f[7] = dev1(ld_h(a.nin[7], o + p - 1, inv_s), wgt(8), a.Rin[o + p - 1], r0);
            } else {
                f[0] = pull_edge_h<1>(a.nin[0], a.nin[opp(1) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[1] = pull_edge_h<2>(a.nin[1], a.nin[opp(2) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[2] = pull_edge_h<3>(a.nin[2], a.nin[opp(3) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[3] = pull_edge_h<4>(a.nin[3], a.nin[opp(4) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[4] = pull_edge_h<5>(a.nin[4], a.nin[opp(5) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[5] = pull_edge_h<6>(a.nin[5], a.nin[opp(6) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[6] = pull_edge_h<7>(a.nin[6], a.nin[opp(7) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                f[7] = pull_edge_h<8>(a.nin[7], a.nin[opp(8) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
            }
            const float dP = pressure_of(f);
            const float it = a.inv_tau[o];
            float F = a.Fp ? a.Fp[o] : 0.0f;
            for (int k = 0; k < a.w.n; ++k)
                if (o == a.w.idx[k])
                    F += a.w.fp[k];
            const float Fq = 0.125f * F;   // w_bar_i = 1/8 (Eq. 3-5a)
            const float keep = 1.0f - it;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                // (1 - 1/tau_f)(a_i - w_i dP) + F~_p/8: Eq. 2-1b relative to R + dP
                const float e = fmaf(-wgt(i + 1), dP, f[i]);
                a.nout[i][o] = __float2half_rn(fmaf(keep, e, Fq) * s);
            }
            a.Rout[o] = r0 + dP;
            if (CHECK) {
                d = dP - dshift;
                q = (r0 - shift) + dP;
                racc.add(d, q);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    nmax = fmaxf(nmax, fabsf(__half2float(a.nout[i][o])));
            }
        }
    }
    if (CHECK) {
        // largest stored magnitude (scaled) seen by this check sweep, for the host's rescale
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1)
            nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, sh));
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned int *>(&a.scale_out[3]), __float_as_uint(nmax));
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
            double sum = 0.0;
            for (int w = 0; w < kBlock / 32; ++w)
                sum += red[w][threadIdx.x];
            a.partials[4 * blockIdx.x + threadIdx.x] = sum;
        }
    }
}


// The FP16 sweep with its input rows staged in shared memory by cp.async.bulk: the
// warp-specialised pipeline of the FP32 staged-rows sweep (producer warp, consumer warps on
// full/empty mbarriers, bounded waits) over 8 FP16 planes (16-byte segments need 8 halo
// values) and the FP32 node-pressure, 1/tau_f (and F~_p) planes (4 halo values).
constexpr int kHaloH = 8;        // FP16 values staged on each side of a strip
constexpr int kHaloF = 4;        // FP32 values staged on each side of a strip
constexpr int kBarBytesH = 128;

template <bool CHECK, int CW, int S>
__global__ void __launch_bounds__(32 * (CW + 1)) k_pressure_rows_h(const __grid_constant__ HalfSweepArgs a,
                                                                   int H)
{
    constexpr int W = 32 * CW;
    constexpr int RWH = W + 2 * kHaloH;            // halves per staged FP16 row
    constexpr int RWF = W + 2 * kHaloF;            // floats per staged FP32 row
    const int nplf = a.Fp ? 3 : 2;                 // FP32 planes staged per row
    const int slot_bytes = 8 * RWH * 2 + nplf * RWF * 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + S;
    unsigned char *ring = smem + kBarBytesH;
    __shared__ double red[CW][4];
    __shared__ float wmax[CW];
    __shared__ int failed;
    const Geom &g = a.g;
    const int p = g.pitch;
    const int strips = (g.nx + W - 1) / W;
    const int x0 = (blockIdx.x % strips) * W;
    const int y0 = (blockIdx.x / strips) * H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (y0 >= g.ny) {
        if (CHECK && threadIdx.x < 4)
            a.partials[4 * blockIdx.x + threadIdx.x] = 0.0;
        return;
    }
    const int y1 = y0 + H < g.ny ? y0 + H : g.ny;
    const int nrows = y1 - y0 + 2;
    const int xah = x0 - kHaloH > 0 ? x0 - kHaloH : 0;
    const int xbh = x0 + W + kHaloH < p ? x0 + W + kHaloH : p;
    const int xaf = x0 - kHaloF > 0 ? x0 - kHaloF : 0;
    const int xbf = x0 + W + kHaloF < p ? x0 + W + kHaloF : p;
    const unsigned segh = (unsigned)(xbh - xah) * 2u, segf = (unsigned)(xbf - xaf) * 4u;
    const int soffh = xah - (x0 - kHaloH), sofff = xaf - (x0 - kHaloF);

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
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nrows; ++t) {
                const int q = t % S;
                if (t >= S && !bar_wait_bounded(empty + q, (unsigned)(t / S - 1) & 1u)) {
                    failed = 1;
                    break;
                }
                const int r = y0 - 1 + t;
                unsigned m = nplf == 3 ? 0x7FFu : 0x3FFu;
                if (r < 0 || r >= g.ny)
                    m = 0u;
                else if (t == 0)
                    m = (1u << 1) | (1u << 4) | (1u << 5) | (1u << 8);
                else if (t == nrows - 1)
                    m = (1u << 3) | (1u << 6) | (1u << 7) | (1u << 8);
                if (!m) {
                    bar_arrive(full + q);
                } else {
                    unsigned bytes = 0;
                    for (int pl = 0; pl < 11; ++pl)
                        if (m & (1u << pl))
                            bytes += pl < 8 ? segh : segf;
                    bar_arrive_tx(full + q, bytes);
                    unsigned char *slot = ring + (size_t)q * slot_bytes;
#pragma unroll
                    for (int pl = 0; pl < 8; ++pl)
                        if (m & (1u << pl))
                            bulk_g2s(slot + (pl * RWH + soffh) * 2, a.nin[pl] + (size_t)r * p + xah,
                                     segh, full + q);
                    float *fslot = reinterpret_cast<float *>(slot + 8 * RWH * 2);
                    if (m & (1u << 8))
                        bulk_g2s(fslot + sofff, a.Rin + (size_t)r * p + xaf, segf, full + q);
                    if (m & (1u << 9))
                        bulk_g2s(fslot + RWF + sofff, a.inv_tau + (size_t)r * p + xaf, segf, full + q);
                    if (m & (1u << 10))
                        bulk_g2s(fslot + 2 * RWF + sofff, a.Fp + (size_t)r * p + xaf, segf, full + q);
                }
                issued = t + 1;
            }
            for (int t = issued - S > 0 ? issued - S : 0; t < issued; ++t)
                bar_wait_bounded(full + t % S, (unsigned)(t / S) & 1u);
        }
    } else {
        const float s = a.scale[0], inv_s = a.scale[1];
        const float shift = CHECK ? a.shift[0] : 0.0f;
        const float dshift = CHECK ? a.shift[1] : 0.0f;
        ResAcc racc;                          // residual sums of this lane over its rows
        float nmax = 0.0f;
        const int col = warp * 32 + lane;
        const int lh = col + kHaloH, lf = col + kHaloF;
        const int x = x0 + col;
        bool ok = true;
        for (int t = 0; t < nrows && ok; ++t) {
            ok = bar_wait_bounded(full + t % S, (unsigned)(t / S) & 1u);
            if (!ok || t < 2)
                continue;
            const int y = y0 - 2 + t;
            const unsigned char *bm = ring + (size_t)((t - 2) % S) * slot_bytes;
            const unsigned char *b0 = ring + (size_t)((t - 1) % S) * slot_bytes;
            const unsigned char *bp = ring + (size_t)(t % S) * slot_bytes;
            const __half *hm = reinterpret_cast<const __half *>(bm);
            const __half *h0 = reinterpret_cast<const __half *>(b0);
            const __half *hp = reinterpret_cast<const __half *>(bp);
            const float *fm = reinterpret_cast<const float *>(bm + 8 * RWH * 2);
            const float *f0 = reinterpret_cast<const float *>(b0 + 8 * RWH * 2);
            const float *fp = reinterpret_cast<const float *>(bp + 8 * RWH * 2);
            float d = 0.0f, q = 0.0f;
            if (x < g.nx) {
                const int o = y * p + x;
                const float r0 = f0[lf];
                float f[8];
                if (interior(g, x, y)) {
                    f[0] = dev1(__half2float(h0[0 * RWH + lh - 1]) * inv_s, wgt(1), f0[lf - 1], r0);
                    f[1] = dev1(__half2float(hm[1 * RWH + lh]) * inv_s, wgt(2), fm[lf], r0);
                    f[2] = dev1(__half2float(h0[2 * RWH + lh + 1]) * inv_s, wgt(3), f0[lf + 1], r0);
                    f[3] = dev1(__half2float(hp[3 * RWH + lh]) * inv_s, wgt(4), fp[lf], r0);
                    f[4] = dev1(__half2float(hm[4 * RWH + lh - 1]) * inv_s, wgt(5), fm[lf - 1], r0);
                    f[5] = dev1(__half2float(hm[5 * RWH + lh + 1]) * inv_s, wgt(6), fm[lf + 1], r0);
                    f[6] = dev1(__half2float(hp[6 * RWH + lh + 1]) * inv_s, wgt(7), fp[lf + 1], r0);
                    f[7] = dev1(__half2float(hp[7 * RWH + lh - 1]) * inv_s, wgt(8), fp[lf - 1], r0);
                } else {
                    f[0] = pull_edge_h<1>(a.nin[0], a.nin[opp(1) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[1] = pull_edge_h<2>(a.nin[1], a.nin[opp(2) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[2] = pull_edge_h<3>(a.nin[2], a.nin[opp(3) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[3] = pull_edge_h<4>(a.nin[3], a.nin[opp(4) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[4] = pull_edge_h<5>(a.nin[4], a.nin[opp(5) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[5] = pull_edge_h<6>(a.nin[5], a.nin[opp(6) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[6] = pull_edge_h<7>(a.nin[6], a.nin[opp(7) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                    f[7] = pull_edge_h<8>(a.nin[7], a.nin[opp(8) - 1], a.Rin, g, a.Pb, x, y, r0, inv_s);
                }
                const float dP = pressure_of(f);
                const float it = f0[RWF + lf];
                float F = a.Fp ? f0[2 * RWF + lf] : 0.0f;
                for (int w = 0; w < a.w.n; ++w)
                    if (o == a.w.idx[w])
                        F += a.w.fp[w];
                const float Fq = 0.125f * F;
                const float keep = 1.0f - it;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float e = fmaf(-wgt(i + 1), dP, f[i]);
                    const __half hv = __float2half_rn(fmaf(keep, e, Fq) * s);
                    a.nout[i][o] = hv;
                    if (CHECK)
                        nmax = fmaxf(nmax, fabsf(__half2float(hv)));
                }
                a.Rout[o] = r0 + dP;
                if (CHECK) {
                    d = dP - dshift;
                    q = (r0 - shift) + dP;
                    racc.add(d, q);
                }
            }
            __syncwarp();
            if (lane == 0)
                bar_arrive(empty + (t - 2) % S);
        }
        if (!ok) {
            failed = 1;
            const __half nan = __float2half(__int_as_float(0x7fc00000));
            if (x < g.nx)
                for (int y = y0; y < y1; ++y)
                    for (int i = 0; i < 8; ++i)
                        a.nout[i][y * p + x] = nan;
        }
        if (CHECK) {
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1)
                nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, sh));
            double v[4];
            racc.warp_totals(v);
            if (lane == 0) {
                red[warp][0] = v[0];
                red[warp][1] = v[1];
                red[warp][2] = v[2];
                red[warp][3] = v[3];
                wmax[warp] = nmax;
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
    if (CHECK && threadIdx.x == 4) {
        float mx = 0.0f;
        for (int w = 0; w < CW; ++w)
            mx = fmaxf(mx, wmax[w]);
        atomicMax(reinterpret_cast<unsigned int *>(&a.scale_out[3]), __float_as_uint(mx));
    }
}

template <int CW, int S>
void *rows_h_func_t(bool check)
{
    return check ? (void *)k_pressure_rows_h<true, CW, S> : (void *)k_pressure_rows_h<false, CW, S>;
}

void *rows_h_func(int width, int slots, bool check)
{
    if (width == 128)
        return rows_h_func_t<4, 8>(check);
    return slots == 6 ? rows_h_func_t<8, 6>(check) : rows_h_func_t<8, 8>(check);
}

}  // namespace
}  // namespace lbm2p_dev

namespace lbm2p_launch {

using namespace lbm2p_dev;

int max_blocks_per_sm_pressure_h()
{
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pressure_h<true>, kBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pressure_h<false>, kBlock, 0);
    const int m = a < b ? a : b;
    return m > 0 ? m : 1;
}

void half_narrow(const HalfConvertArgs &a, int grid, void *stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_absmax<<<grid, kBlock, 0, st>>>(a);
    k_set_scale<<<1, 1, 0, st>>>(a.scale);
    k_narrow<<<grid, kBlock, 0, st>>>(a);
}

void half_rescale(const HalfConvertArgs &a, float factor, int grid, void *stream)
{
    k_rescale<<<grid, kBlock, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a, factor);
}

void half_widen(const HalfConvertArgs &a, int grid, void *stream)
{
    k_widen<<<grid, kBlock, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
}

void pressure_sweep_h(const HalfSweepArgs &a, bool check, int grid, void *stream)
{
    void *args[] = {(void *)&a};
    cudaLaunchKernel(check ? (void *)k_pressure_h<true> : (void *)k_pressure_h<false>, dim3(grid),
                     dim3(kBlock), args, 0, reinterpret_cast<cudaStream_t>(stream));
}

size_t rows_h_smem_bytes(int width, int slots, bool has_fp)
{
    const size_t slot = 8 * (size_t)(width + 2 * kHaloH) * 2 +
                        (size_t)(has_fp ? 3 : 2) * (width + 2 * kHaloF) * 4;
    return 128 + kBarBytesH + (size_t)slots * slot;
}

cudaError_t rows_h_prepare(int width, int slots)
{
    const int bytes = (int)rows_h_smem_bytes(width, slots, true);
    for (bool c : {false, true}) {
        cudaError_t e = cudaFuncSetAttribute(rows_h_func(width, slots, c),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

int rows_h_blocks_per_sm(int width, int slots, bool has_fp)
{
    int lo = 1 << 30;
    for (bool c : {false, true}) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rows_h_func(width, slots, c), width + 32,
                                                      rows_h_smem_bytes(width, slots, has_fp));
        lo = b < lo ? b : lo;
    }
    return lo;
}

void pressure_sweep_rows_h(const HalfSweepArgs &a, bool check, int width, int slots, int H,
                           int grid, void *stream)
{
    void *args[] = {(void *)&a, (void *)&H};
    cudaLaunchKernel(rows_h_func(width, slots, check), dim3(grid), dim3(width + 32), args,
                     rows_h_smem_bytes(width, slots, a.Fp != nullptr),
                     reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace lbm2p_launch
