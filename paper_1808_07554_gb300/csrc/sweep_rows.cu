// Pressure sweep (Eq. 3-1, pull stream + BGK collide) with its input rows staged in shared
// memory by the bulk-copy engine.
//
// A block owns a strip of W = BT * NPT columns and a chunk of H rows, and marches down the
// chunk.  Pulling into row y reads populations of rows y-1 (directions with c_y = +1),
// y (c_y = 0) and y+1 (c_y = -1), the reference pressure R of all three rows, and 1/tau_f
// and F~_p of row y.  Each input row r is therefore copied once, as row segments
// [x0 - 4, x0 + W + 4) of every plane (16-byte aligned, clamped to the row), by one
// cp.async.bulk per plane into a ring of kRowsSlots slots; kRowsDepth rows are in flight
// while the block computes, and every copy completes on the slot's mbarrier.  The
// arithmetic of an interior node is that of gather_a / sweep_node with the loads taken
// from shared memory; edge nodes take the global-memory gather with the wall rules.  The
// populations written are bit-identical to the other single-sweep kernels.
//
// Every wait on an mbarrier is bounded: a block that gives up waits (bounded) for its own
// copies still in flight, writes NaN into its outputs and residual partials, and returns,
// so the host sees a non-finite residual instead of a hung GPU.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm2p_device.cuh"
#include "lbm2p_node.cuh"

namespace lbm2p_dev {
namespace {

constexpr int kRowsDepth = 4;                 // input rows in flight
constexpr int kRowsSlots = kRowsDepth + 2;    // plus the two rows behind the newest one
constexpr int kRowsPlanes = 11;               // n_1..n_8, R, 1/tau_f, F~_p
constexpr int kRowsHalo = 4;                  // floats staged on each side of the strip
constexpr int kRowsBarBytes = 128;            // mbarriers at the start of shared memory
constexpr unsigned kWaitLimit = 1u << 22;     // try_wait polls before a block gives up

__device__ __forceinline__ unsigned smem_u32(const void *ptr)
{
    return (unsigned)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void bar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bar_arrive_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (bar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(float *dst, const float *src, unsigned bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <bool CHECK, bool WRITE_P, int BT, int NPT>
__global__ void __launch_bounds__(BT) k_pressure_rows(const __grid_constant__ PressureArgs a, int H)
{
    constexpr int W = BT * NPT;
    constexpr int RW = W + 2 * kRowsHalo;          // floats per staged plane row
    constexpr int SLOT = kRowsPlanes * RW;         // floats per ring slot
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk copies need 16-byte aligned destinations: align the ring explicitly (the launch
    // adds 128 bytes of slack for this)
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float *ring = reinterpret_cast<float *>(smem + kRowsBarBytes);
    const Geom &g = a.g;
    const int p = g.pitch;
    const int strips = (g.nx + W - 1) / W;
    const int x0 = (blockIdx.x % strips) * W;
    const int y0 = (blockIdx.x / strips) * H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red[BT / 32][4];
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
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
    const float shift = CHECK ? a.shift[0] : 0.0f;
    const float dshift = CHECK ? a.shift[1] : 0.0f;

    // planes of input row t (y0 - 1 + t): the first row feeds only the c_y = +1 pulls of
    // row y0, the last only the c_y = -1 pulls of row y1 - 1; both also give R
    auto row_mask = [&](int t) -> unsigned {
        const int r = y0 - 1 + t;
        if (r < 0 || r >= g.ny)
            return 0u;
        if (t == 0)
            return (1u << 1) | (1u << 4) | (1u << 5) | (1u << 8);
        if (t == nrows - 1)
            return (1u << 3) | (1u << 6) | (1u << 7) | (1u << 8);
        return a.Fp ? 0x7FFu : 0x3FFu;
    };
    auto plane_src = [&](int q) -> const float * {
        return q < 8 ? a.fin[q] : (q == 8 ? a.R : (q == 9 ? a.inv_tau : a.Fp));
    };
    auto issue = [&](int t) {                      // thread 0 only
        const int s = t % kRowsSlots;
        const unsigned m = row_mask(t);
        if (!m) {
            bar_arrive(bar + s);
            return;
        }
        bar_arrive_tx(bar + s, (unsigned)__popc(m) * seg);
        const size_t roff = (size_t)(y0 - 1 + t) * p + xa;
        float *slot = ring + (size_t)s * SLOT + soff;
#pragma unroll
        for (int q = 0; q < kRowsPlanes; ++q)
            if (m & (1u << q))
                bulk_g2s(slot + q * RW, plane_src(q) + roff, seg, bar + s);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRowsSlots; ++s)
            bar_init(bar + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 0; t < kRowsDepth && t < nrows; ++t)
            issue(t);

    int failed_at = -1;
    for (int t = 0; t < nrows; ++t) {
        const bool ok = bar_wait_bounded(bar + t % kRowsSlots, (unsigned)(t / kRowsSlots) & 1u);
        if (t >= 2) {
            // output row y = y0 - 2 + t from input rows y - 1, y, y + 1
            const int y = y0 - 2 + t;
            const float *sm = ring + (size_t)((t - 2) % kRowsSlots) * SLOT;
            const float *s0 = ring + (size_t)((t - 1) % kRowsSlots) * SLOT;
            const float *sp = ring + (size_t)(t % kRowsSlots) * SLOT;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int lx = (int)threadIdx.x + k * BT + kRowsHalo;
                const int x = x0 + lx - kRowsHalo;
                float d = 0.0f, q = 0.0f;
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
                    if (CHECK) {
                        d = (dP - a.Pio[o]) - dshift;
                        q = (r0 - shift) + dP;
                    }
                    if (WRITE_P)
                        a.Pio[o] = dP;
                }
                if (CHECK) {
                    const float s0s = warp_sum(d), s1s = warp_sum(d * d);
                    const float s2s = warp_sum(q), s3s = warp_sum(q * q);
                    if (lane == 0) {
                        acc0 += s0s;
                        acc1 += s1s;
                        acc2 += s2s;
                        acc3 += s3s;
                    }
                }
            }
        }
        // every thread is done with input row t - 2 before its slot is refilled
        if (__syncthreads_or(!ok)) {
            failed_at = t;
            break;
        }
        if (threadIdx.x == 0 && t + kRowsDepth < nrows)
            issue(t + kRowsDepth);
    }

    if (failed_at >= 0) {
        // rows failed_at .. failed_at + depth - 1 may still be arriving: wait for them
        // (bounded), then poison this block's part of the sweep
        if (threadIdx.x == 0)
            for (int t = failed_at; t < nrows && t < failed_at + kRowsDepth; ++t)
                bar_wait_bounded(bar + t % kRowsSlots, (unsigned)(t / kRowsSlots) & 1u);
        __syncthreads();
        const float nan = __int_as_float(0x7fc00000);
        for (int y = y0; y < y1; ++y)
            for (int k = 0; k < NPT; ++k) {
                const int x = x0 + (int)threadIdx.x + k * BT;
                if (x < g.nx)
                    for (int i = 0; i < 8; ++i)
                        a.fout[i][y * p + x] = nan;
            }
        if (CHECK && threadIdx.x < 4)
            a.partials[4 * blockIdx.x + threadIdx.x] = (double)nan;
        return;
    }

    if (CHECK) {
        if (lane == 0) {
            red[warp][0] = acc0;
            red[warp][1] = acc1;
            red[warp][2] = acc2;
            red[warp][3] = acc3;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int w = 0; w < BT / 32; ++w)
                s += red[w][threadIdx.x];
            a.partials[4 * blockIdx.x + threadIdx.x] = s;
        }
    }
}

template <int BT, int NPT>
void *rows_func_t(bool check, bool write_p)
{
    return check ? (write_p ? (void *)k_pressure_rows<true, true, BT, NPT>
                            : (void *)k_pressure_rows<true, false, BT, NPT>)
                 : (write_p ? (void *)k_pressure_rows<false, true, BT, NPT>
                            : (void *)k_pressure_rows<false, false, BT, NPT>);
}

void *rows_func(int bt, int npt, bool check, bool write_p)
{
    if (bt == 128)
        return rows_func_t<128, 1>(check, write_p);
    if (npt == 2)
        return rows_func_t<256, 2>(check, write_p);
    return rows_func_t<256, 1>(check, write_p);
}

}  // namespace
}  // namespace lbm2p_dev

namespace lbm2p_launch {

using lbm2p_dev::PressureArgs;

bool rows_shape_ok(int bt, int npt)
{
    return (bt == 128 && npt == 1) || (bt == 256 && (npt == 1 || npt == 2));
}

size_t rows_smem_bytes(int bt, int npt)
{
    const size_t rw = (size_t)bt * npt + 2 * lbm2p_dev::kRowsHalo;
    return 128 + lbm2p_dev::kRowsBarBytes +
           (size_t)lbm2p_dev::kRowsSlots * lbm2p_dev::kRowsPlanes * rw * sizeof(float);
}

long long rows_grid(int bt, int npt, int H, int nx, int ny)
{
    const int W = bt * npt;
    return (long long)((nx + W - 1) / W) * ((ny + H - 1) / H);
}

cudaError_t rows_prepare(int bt, int npt)
{
    const int bytes = (int)rows_smem_bytes(bt, npt);
    for (bool c : {false, true})
        for (bool w : {false, true}) {
            cudaError_t e = cudaFuncSetAttribute(lbm2p_dev::rows_func(bt, npt, c, w),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess)
                return e;
        }
    return cudaSuccess;
}

int rows_blocks_per_sm(int bt, int npt)
{
    int lo = 1 << 30;
    for (bool c : {false, true})
        for (bool w : {false, true}) {
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lbm2p_dev::rows_func(bt, npt, c, w),
                                                          bt, rows_smem_bytes(bt, npt));
            lo = b < lo ? b : lo;
        }
    return lo;
}

void pressure_sweep_rows(const PressureArgs &a, bool check, bool write_p, int bt, int npt, int H,
                         int grid, void *stream)
{
    void *args[] = {(void *)&a, (void *)&H};
    cudaLaunchKernel(lbm2p_dev::rows_func(bt, npt, check, write_p), dim3(grid), dim3(bt), args,
                     rows_smem_bytes(bt, npt), reinterpret_cast<cudaStream_t>(stream));
}

cudaError_t node_pressure_rows(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep,
                               const PressureArgs &a, bool check, bool write_p, int bt, int npt,
                               int H, int grid)
{
    cudaKernelNodeParams prm{};
    prm.func = lbm2p_dev::rows_func(bt, npt, check, write_p);
    prm.gridDim = dim3((unsigned)grid);
    prm.blockDim = dim3((unsigned)bt);
    prm.sharedMemBytes = (unsigned)rows_smem_bytes(bt, npt);
    void *args[] = {(void *)&a, (void *)&H};
    prm.kernelParams = args;
    prm.extra = nullptr;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &prm);
}

}  // namespace lbm2p_launch
