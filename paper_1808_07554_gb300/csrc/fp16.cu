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
            a.R[o] = a.Rh[o];
        }
    }
}

template <bool CHECK>
__global__ void __launch_bounds__(kBlock) k_pressure_h(const __grid_constant__ HalfSweepArgs a)
{
    const Geom &g = a.g;
    const int lane = threadIdx.x & 31;
    const float s = a.scale[0], inv_s = a.scale[1];
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
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
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    nmax = fmaxf(nmax, fabsf(__half2float(a.nout[i][o])));
            }
        }
        if (CHECK) {
            const float s0 = warp_sum(d), s1 = warp_sum(d * d), s2 = warp_sum(q), s3 = warp_sum(q * q);
            if (lane == 0) {
                acc0 += s0;
                acc1 += s1;
                acc2 += s2;
                acc3 += s3;
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
        if (lane == 0) {
            red[warp][0] = acc0;
            red[warp][1] = acc1;
            red[warp][2] = acc2;
            red[warp][3] = acc3;
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

}  // namespace lbm2p_launch
