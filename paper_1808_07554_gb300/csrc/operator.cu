// A small convolutional operator on the fifth-generation tensor cores (tcgen05): the 3x3
// convolutions of a five-layer network that predicts the next step's pressure for the warm
// start of the lattice Boltzmann pressure solve, with the kernels its training needs.
//
// Convolution as an implicit GEMM (forward and input gradient): a CTA computes tiles of
// M = 128 consecutive pixels by N = C_out channels; the reduction runs over K = 9 taps x C_in
// channels in steps of 16.  For each K-step every thread gathers 16 bytes (8 channels of one
// pixel at one tap, zero outside the image) into a shared-memory stage laid out as the
// tensor core's K-major core matrices (8 rows x 16 bytes each); thread 0 issues one
// tcgen05.mma (M = 128, N = C_out, K = 16, BF16 inputs, FP32 accumulator in tensor memory)
// and commits it to the stage's mbarrier, which frees the stage for the K-step NS later.
// The weights of all K-steps stay in shared memory for the whole kernel.  After a tile's
// last K-step the CTA waits for its MMAs, reads the accumulator with tcgen05.ld (each warp
// its 32 tensor-memory lanes, i.e. its 32 pixels), adds the bias, applies the activation
// (and the ReLU mask of the input-gradient pass) and stores BF16 channels-last rows.
//
// Weight gradient: M = 128 rows of (tap, input channel), N = C_out, K = pixels; the stage
// loader transposes 16-pixel chunks of the channels-last activations and output gradients
// into K-major core matrices; each CTA reduces a share of the pixels and adds its partial
// sums into the FP32 gradient with atomics.
//
// Every wait on an mbarrier is bounded; a CTA that gives up records the failure in *err,
// waits (bounded) for its MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm2p.h"
#include "lbm2p_async.cuh"
#include "lbm2p_operator.h"

namespace lbm2p_internal {
lbm2p_status set_global_error(lbm2p_status st, const char *fmt, ...);
}

namespace lbm2p_op {
using lbm2p_dev::bar_init;
using lbm2p_dev::bar_try_wait;
using lbm2p_dev::kWaitLimit;
using lbm2p_dev::smem_u32;

typedef __nv_bfloat16 bf16;

// ---- tcgen05 primitives (inline PTX) --------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory writes of this thread become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D (tensor memory) = A B^T (+ D when accumulate), A: M x 16, B: N x 16, both K-major
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the mbarrier receives one arrival when every tcgen05.mma issued so far by this thread is done
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 tensor-memory lanes x 16 consecutive 32-bit columns: thread l of the warp receives lane
// (base lane + l); the wait for the load is part of the same statement
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle, K-major core matrices of 8 rows x 16 bytes:
// start address, LBO = bytes between the two core matrices along K, SBO = bytes between
// 8-row groups along M (or N); bits 46..48 hold the descriptor version 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bit 4), BF16 A and B (bits 7, 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (bar_try_wait(bar, parity))
            return true;
    return false;
}

constexpr int kThreads = 256;
constexpr int kStages = 4;
constexpr uint32_t kABytes = 128 * 16 * 2;       // one A stage: 128 rows x 16 BF16
constexpr uint32_t kTmemCols = 32;

struct ConvArgs {
    const bf16 *x;        // [npix][cin]
    const bf16 *w;        // [9][cout][cin]
    const float *bias;    // [cout] or null
    const bf16 *mask;     // [npix][cout] or null
    bf16 *y;              // [npix][cout] or null
    float *y0;            // [npix] or null
    int nimg, H, W;
    int act;
    int *err;
};

// ---- convolution on staged rows ----------------------------------------------------------
// A tile is 128 consecutive pixels of one image row (x0 .. x0 + 127, the last tile of a row
// ragged).  Its three input rows y - 1 .. y + 1, pixels x0 - 1 .. x0 + 128, are copied once into
// shared memory as channel-chunk planes: chunk c (channels 8 c .. 8 c + 7) of staged row r is
// an array of 130 pixels x 16 bytes.  In that layout the A operand of tap (dy, dx) and K-half j
// is the K-major core-matrix matrix that starts at row dy + 1, chunk 2 j, pixel dx + 1: a shift
// by one pixel is a shift of the descriptor's start address by 16 bytes, so all 9 x C_in / 16
// MMAs of a tile read the same staged rows.  Two stage buffers: the rows of the next tile are
// copied while the tensor core works on the current one.
constexpr int kRowPix = 130;                        // staged pixels per row
constexpr uint32_t kChunkBytes = kRowPix * 16;      // one channel chunk of a staged row

template <int CIN, int COUT>
constexpr size_t conv_rows_smem_bytes()
{
    return (size_t)(9 * CIN / 16) * COUT * 32 + 2 * (size_t)3 * (CIN / 8) * kChunkBytes + 8 + 16 + 128;
}

// 16 bytes global -> shared without a register round trip (cp.async); a source outside the
// image (valid false) reads nothing and fills zeros.  Complete after cp_async_wait_all.
__device__ __forceinline__ void cp_async16(unsigned char *dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// the three input rows of a tile into a stage buffer (asynchronous: every copy is in flight
// at once; the caller waits with cp_async_wait_all)
template <int CIN, int COUT>
__device__ __forceinline__ void stage_rows(const ConvArgs &a, unsigned char *buf, long long tile,
                                           int tiles_x, int tid)
{
    constexpr int CH = CIN / 8;
    const int img = (int)(tile / ((long long)a.H * tiles_x));
    const int rem = (int)(tile - (long long)img * a.H * tiles_x);
    const int y = rem / tiles_x, x0 = (rem - y * tiles_x) * 128;
    for (int i = tid; i < 3 * kRowPix * CH; i += kThreads) {
        const int c = i % CH, px = (i / CH) % kRowPix, r = i / (CH * kRowPix);
        const int yy = y + r - 1, xx = x0 + px - 1;
        const bool valid = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        const bf16 *src = valid ? a.x + (((size_t)img * a.H + yy) * a.W + xx) * CIN + 8 * c : a.x;
        cp_async16(buf + (r * CH + c) * kChunkBytes + px * 16, src, valid);
    }
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) k_conv3x3_rows(const ConvArgs a)
{
    constexpr int CH = CIN / 8;
    constexpr int KH = CIN / 16;                      // K-halves of 16 channels per tap
    constexpr int KS = 9 * KH;
    constexpr uint32_t kBBytes = COUT * 16 * 2;
    constexpr uint32_t kStageBytes = 3 * CH * kChunkBytes;
    constexpr uint32_t IDESC = idesc_bf16(128, COUT);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    unsigned char *wsm = smem;
    unsigned char *stg = smem + KS * kBBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(stg + 2 * kStageBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < KS * COUT * 2; i += kThreads) {
        const int s = i / (COUT * 2), rem = i - s * (COUT * 2);
        const int kc = rem / COUT, n = rem - kc * COUT;
        const int t = s / KH, j = s - t * KH;
        const uint4 v = *reinterpret_cast<const uint4 *>(a.w + ((size_t)(t * COUT + n) * CIN + 16 * j + 8 * kc));
        *reinterpret_cast<uint4 *>(wsm + s * kBBytes + kc * (COUT * 16) + n * 16) = v;
    }
    if (warp == 0) {
        tmem_alloc(tslot, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int tiles_x = (a.W + 127) / 128;
    const long long tiles = (long long)a.nimg * a.H * tiles_x;
    long long tile = blockIdx.x;
    if (tile < tiles)
        stage_rows<CIN, COUT>(a, stg, tile, tiles_x, tid);
    cp_async_wait_all();
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    unsigned phase = 0;
    int b = 0;
    bool ok = true;
    for (; tile < tiles; tile += gridDim.x, b ^= 1) {
        unsigned char *cur = stg + b * kStageBytes;
        if (tid == 0) {
            tc_fence_after();
            int s = 0;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
#pragma unroll
                for (int j = 0; j < KH; ++j, ++s) {
                    const uint32_t start = smem_u32(cur + ((t / 3) * CH + 2 * j) * kChunkBytes +
                                                    (t % 3) * 16);
                    const uint64_t ad = sdesc(start, kChunkBytes, 128);
                    const uint64_t bd = sdesc(smem_u32(wsm + s * kBBytes), COUT * 16, 128);
                    umma_bf16(tmem, ad, bd, IDESC, s > 0 ? 1u : 0u);
                }
            }
            umma_commit(bar);
        }
        // the next tile's rows into the other buffer while the tensor core works
        const long long next = tile + gridDim.x;
        if (next < tiles)
            stage_rows<CIN, COUT>(a, stg + (b ^ 1) * kStageBytes, next, tiles_x, tid);
        if (!wait_bounded(bar, phase)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        const int img = (int)(tile / ((long long)a.H * tiles_x));
        const int rem = (int)(tile - (long long)img * a.H * tiles_x);
        const int y = rem / tiles_x, x0 = (rem - y * tiles_x) * 128;
        const int cb = 16 * (warp >> 2);
        if (cb < COUT) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb, v);
            const int x = x0 + 32 * (warp & 3) + lane;
            if (x < a.W) {
                const long long q = ((long long)img * a.H + y) * a.W + x;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float u = v[i] + (a.bias ? a.bias[cb + i] : 0.0f);
                    if (a.act == 1)
                        u = fmaxf(u, 0.0f);
                    v[i] = u;
                }
                if (a.mask) {
                    const bf16 *mk = a.mask + q * COUT + cb;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (!(__bfloat162float(mk[i]) > 0.0f))
                            v[i] = 0.0f;
                }
                if (a.y) {
                    __align__(16) bf16 o[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        o[i] = __float2bfloat16_rn(v[i]);
                    uint4 *dst = reinterpret_cast<uint4 *>(a.y + q * COUT + cb);
                    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
                    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
                }
                if (a.y0 && cb == 0)
                    a.y0[q] = v[0];
            }
        }
        // the next tile's rows are in place, and the accumulator and the buffer just read are
        // free, once every thread is past here
        cp_async_wait_all();
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    }
    cp_async_wait_all();
    if (!ok) {
        if (tid == 0)
            atomicExch(a.err, 1);
        wait_bounded(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ---- weight gradient --------------------------------------------------------------------
struct WgradArgs {
    const bf16 *x;        // [npix][cin]
    const bf16 *g;        // [npix][cout]
    float *dw;            // [9][cout][cin]
    int nimg, H, W;
    int *err;
};

template <int CIN, int COUT>
constexpr size_t wgrad_smem_bytes()
{
    return (size_t)kStages * (kABytes + COUT * 32) + kStages * 8 + 16 + 128;
}

// grid (M-tiles of 128 (tap, channel) rows, pixel splits): CTA (mt, sp) reduces the K-steps
// sp, sp + gridDim.y, ... of 16 pixels each
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) k_conv3x3_wgrad(const WgradArgs a)
{
    constexpr uint32_t kBBytes = COUT * 16 * 2;
    constexpr uint32_t IDESC = idesc_bf16(128, COUT);
    constexpr int R = 9 * CIN;                         // rows (tap, ci)
    constexpr int TPT = 128 / CIN;                     // taps per M-tile
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    unsigned char *asm_ = smem;
    unsigned char *bsm = smem + kStages * kABytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(bsm + kStages * kBBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x;
    const int t0 = mt * TPT;                           // first tap of this M-tile

    if (warp == 0) {
        tmem_alloc(tslot, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s)
            bar_init(bars + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const long long hw = (long long)a.H * a.W;
    const long long npix = (long long)a.nimg * hw;
    const long long ksteps = (npix + 15) / 16;
    unsigned gstep = 0;
    bool ok = true;
    // loader roles: A: thread -> (pixel k = tid % 16, tap slot u, channel chunk c): 16 x TPT x
    // (CIN / 8) = 256 items; B: threads 0 .. 2 COUT - 1 -> (pixel k, channel chunk of g)
    const int k = tid & 15;
    const int item = tid >> 4;                         // 0 .. 15
    const int u = item / (CIN / 8), c = item - u * (CIN / 8);
    for (long long ks = blockIdx.y; ks < ksteps; ks += gridDim.y, ++gstep) {
        const int st = (int)(gstep % kStages);
        if (gstep >= (unsigned)kStages && !wait_bounded(bars + st, ((gstep / kStages) + 1u) & 1u)) {
            ok = false;
            break;
        }
        unsigned char *As = asm_ + st * kABytes;
        unsigned char *Bs = bsm + st * kBBytes;
        const long long p = ks * 16 + k;
        int img = 0, y = 0, x = 0;
        if (p < npix) {
            img = (int)(p / hw);
            const int r = (int)(p - (long long)img * hw);
            y = r / a.W;
            x = r - y * a.W;
        }
        // A row m = u * CIN + 8 c + e holds x[p + d_t][8 c + e], t = t0 + u (zero past row R)
        {
            const int t = t0 + u;
            const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
            __align__(16) bf16 v[8];
            *reinterpret_cast<uint4 *>(v) = make_uint4(0u, 0u, 0u, 0u);
            if (t < 9 && p < npix && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(
                    a.x + (((size_t)img * a.H + yy) * a.W + xx) * CIN + 8 * c);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int mrow = u * CIN + 8 * c + e;
                *reinterpret_cast<bf16 *>(As + (k >> 3) * 2048 + mrow * 16 + (k & 7) * 2) = v[e];
            }
        }
        // B row n = 8 c + e holds g[p][8 c + e]
        if (tid < 16 * (COUT / 8)) {
            const int cb = tid >> 4;
            __align__(16) bf16 v[8];
            *reinterpret_cast<uint4 *>(v) = make_uint4(0u, 0u, 0u, 0u);
            if (p < npix)
                *reinterpret_cast<uint4 *>(v) =
                    *reinterpret_cast<const uint4 *>(a.g + p * COUT + 8 * cb);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int n = 8 * cb + e;
                *reinterpret_cast<bf16 *>(Bs + (k >> 3) * (COUT * 16) + n * 16 + (k & 7) * 2) = v[e];
            }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint64_t ad = sdesc(smem_u32(As), 2048, 128);
            const uint64_t bd = sdesc(smem_u32(Bs), COUT * 16, 128);
            umma_bf16(tmem, ad, bd, IDESC, gstep > 0 ? 1u : 0u);
            umma_commit(bars + st);
        }
    }
    if (ok && gstep > 0) {
        const unsigned last = gstep - 1;
        if (!wait_bounded(bars + last % kStages, (last / kStages) & 1u))
            ok = false;
    }
    if (ok && gstep > 0) {
        tc_fence_after();
        const int cb = 16 * (warp >> 2);
        if (cb < COUT) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb, v);
            const int row = mt * 128 + 32 * (warp & 3) + lane;
            if (row < R) {
                const int t = row / CIN, ci = row - t * CIN;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    atomicAdd(a.dw + ((size_t)t * COUT + cb + i) * CIN + ci, v[i]);
            }
        }
    }
    if (!ok) {
        if (tid == 0)
            atomicExch(a.err, 1);
        if (gstep > 0)
            wait_bounded(bars + (gstep - 1) % kStages, ((gstep - 1) / kStages) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ---- CUDA-core helpers -------------------------------------------------------------------
__global__ void k_bias_grad(const bf16 *g, float *db, long long npix, int cout)
{
    // one block per channel group of 32 pixels strided; thread -> channel (tid % cout)
    __shared__ float acc[32];
    const int c = threadIdx.x % cout;
    const int lanes = blockDim.x / cout;
    const int l = threadIdx.x / cout;
    float s = 0.0f;
    for (long long p = (long long)blockIdx.x * lanes + l; p < npix; p += (long long)gridDim.x * lanes)
        s += __bfloat162float(g[p * cout + c]);
    if (threadIdx.x < cout)
        acc[threadIdx.x] = 0.0f;
    __syncthreads();
    atomicAdd(&acc[c], s);
    __syncthreads();
    if (threadIdx.x < cout)
        atomicAdd(db + threadIdx.x, acc[threadIdx.x]);
}

__global__ void k_flip(const bf16 *w, bf16 *wt, int cin, int cout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // over wt[t][ci][co]
    if (i >= 9 * cin * cout)
        return;
    const int t = i / (cin * cout), r = i - t * cin * cout;
    const int ci = r / cout, co = r - ci * cout;
    wt[i] = w[((size_t)(8 - t) * cout + co) * cin + ci];
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, bf16 *pb, long long n,
                       float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (pb)
            pb[i] = __float2bfloat16_rn(pi);
    }
}

__device__ __forceinline__ float sd_of(const double *st, long long n)
{
    const double m = st[0] / (double)n;
    const double v = st[1] / (double)n - m * m;
    return v > 1e-60 ? (float)sqrt(v) : 1.0f;
}

__global__ void k_diff_stats(const float *a, const float *b, long long n, double *st)
{
    __shared__ double red[2][8];
    double s1 = 0.0, s2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)b[i];
        s1 += d;
        s2 += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        atomicAdd(st, t1);
        atomicAdd(st + 1, t2);
    }
}

__global__ void k_features(const float *lnK, const float *S, const float *Sp, const float *P,
                           const float *Pp, const double *dss, const double *dps, bf16 *feat,
                           long long n, float sm, float ss)
{
    const float inv_ds = 1.0f / sd_of(dss, n), inv_dp = 1.0f / sd_of(dps, n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        __align__(16) bf16 o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c)
            o[c] = __float2bfloat16_rn(0.0f);
        o[0] = __float2bfloat16_rn(lnK[i]);
        o[1] = __float2bfloat16_rn((S[i] - sm) / ss);
        o[2] = __float2bfloat16_rn((S[i] - Sp[i]) * inv_ds);
        o[3] = __float2bfloat16_rn((P[i] - Pp[i]) * inv_dp);
        uint4 *dst = reinterpret_cast<uint4 *>(feat + i * 16);
        dst[0] = reinterpret_cast<const uint4 *>(o)[0];
        dst[1] = reinterpret_cast<const uint4 *>(o)[1];
    }
}

__global__ void k_target(const float *Pn, const float *P, const float *Pp, const double *dps,
                         float *out, long long n)
{
    const float inv_dp = 1.0f / sd_of(dps, n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (Pn[i] - (2.0f * P[i] - Pp[i])) * inv_dp;
}

__global__ void k_predict(const float *P, const float *Pp, const float *d, const double *dps,
                          float *out, long long n)
{
    const float sd = sd_of(dps, n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (2.0f * P[i] - Pp[i]) + sd * d[i];
}

__global__ void k_mse_grad(const float *y0, const float *t, bf16 *g, double *loss, long long n,
                           int cout)
{
    __shared__ double red[8];
    double s = 0.0;
    const float sc = 2.0f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float e = y0[i] - t[i];
        s += (double)e * e;
        g[i * cout] = __float2bfloat16_rn(sc * e);
        for (int c = 1; c < cout; ++c)
            g[i * cout + c] = __float2bfloat16_rn(0.0f);
    }
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            tot += red[w];
        atomicAdd(loss, tot / (double)n);
    }
}

// ---- launch helpers -----------------------------------------------------------------------
int g_sms = 0;

int sm_count()
{
    if (g_sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            g_sms = 1;
    }
    return g_sms;
}

// CTAs of `func` that fit on one SM by its registers, threads and `smem` bytes of dynamic
// shared memory (the occupancy rule written out from the device attributes), and by the tensor
// memory (kTmemCols of the 512 columns per CTA)
int resident_per_sm(const void *func, size_t smem)
{
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, func) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 1;
    const long long per_smem = (long long)smem_sm / ((long long)smem + fa.sharedSizeBytes + reserved);
    const int regs_cta = ((fa.numRegs * 32 + 255) / 256) * 256 * (kThreads / 32);
    const long long per_regs = regs_cta > 0 ? regs_sm / regs_cta : 1;
    long long per = per_smem < per_regs ? per_smem : per_regs;
    per = per < thr_sm / kThreads ? per : thr_sm / kThreads;
    per = per < 512 / (long long)kTmemCols ? per : 512 / (long long)kTmemCols;
    return per < 1 ? 1 : (int)per;
}

template <int CIN, int COUT>
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t s)
{
    const size_t smem = conv_rows_smem_bytes<CIN, COUT>();
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_rows<CIN, COUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1/shared storage as shared memory, so that several CTAs (each ~69 KB
    // for 32 input channels) fit on an SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv3x3_rows<CIN, COUT>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess)
        return e;
    // the runtime's occupancy query answered one CTA per SM for this kernel, where its
    // registers and shared memory allow three (ncu's occupancy limits agree with the latter)
    const int per_sm = resident_per_sm((const void *)k_conv3x3_rows<CIN, COUT>, smem);
    const long long tiles = (long long)a.nimg * a.H * ((a.W + 127) / 128);
    long long grid = (long long)sm_count() * per_sm;
    if (grid > tiles)
        grid = tiles;
    k_conv3x3_rows<CIN, COUT><<<(unsigned)grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t s)
{
    const size_t smem = wgrad_smem_bytes<CIN, COUT>();
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_wgrad<CIN, COUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv3x3_wgrad<CIN, COUT>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3x3_wgrad<CIN, COUT>, kThreads,
                                                      smem);
    if (e != cudaSuccess)
        return e;
    per_sm = per_sm < 1 ? 1 : (per_sm > 512 / (int)kTmemCols ? 512 / (int)kTmemCols : per_sm);
    const int mtiles = (9 * CIN + 127) / 128;
    const long long ksteps = ((long long)a.nimg * a.H * a.W + 15) / 16;
    long long splits = (long long)sm_count() * per_sm / mtiles;
    if (splits < 1)
        splits = 1;
    if (splits > ksteps)
        splits = ksteps;
    if (splits > 65535)
        splits = 65535;
    k_conv3x3_wgrad<CIN, COUT><<<dim3((unsigned)mtiles, (unsigned)splits), kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool shape_ok(int n_img, int H, int W, int c_in, int c_out)
{
    return n_img >= 1 && H >= 1 && W >= 1 && (c_in == 16 || c_in == 32) &&
           (c_out == 16 || c_out == 32) && (long long)n_img * H * W < (1LL << 40);
}

unsigned grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    const long long cap = (long long)sm_count() * 16;
    if (b > cap)
        b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace lbm2p_op

using namespace lbm2p_op;
using lbm2p_internal::set_global_error;

extern "C" {

lbm2p_status lbm2p_op_conv3x3(const void *x, const void *w, const float *bias, const void *mask,
                              void *y, float *y0, int n_img, int H, int W, int c_in, int c_out,
                              int act, int *err, void *stream)
{
    if (!shape_ok(n_img, H, W, c_in, c_out))
        return set_global_error(LBM2P_EINVAL, "conv3x3: need n_img, H, W >= 1 and C_in, C_out in {16, 32}");
    if (!x || !w || !err || (!y && !y0) || act < 0 || act > 1)
        return set_global_error(LBM2P_EINVAL, "conv3x3: x, w, err and one of y, y0 are required; act 0 or 1");
    if (!aligned16(x) || !aligned16(w) || (y && !aligned16(y)) || (mask && !aligned16(mask)))
        return set_global_error(LBM2P_EINVAL, "conv3x3: x, w, y and mask must be 16-byte aligned");
    if (y && (y == x || y == mask))
        return set_global_error(LBM2P_EINVAL, "conv3x3: y must not alias x or mask");
    ConvArgs a{};
    a.x = static_cast<const bf16 *>(x);
    a.w = static_cast<const bf16 *>(w);
    a.bias = bias;
    a.mask = static_cast<const bf16 *>(mask);
    a.y = static_cast<bf16 *>(y);
    a.y0 = y0;
    a.nimg = n_img;
    a.H = H;
    a.W = W;
    a.act = act;
    a.err = err;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (c_in == 16)
        e = c_out == 16 ? launch_conv<16, 16>(a, s) : launch_conv<16, 32>(a, s);
    else
        e = c_out == 16 ? launch_conv<32, 16>(a, s) : launch_conv<32, 32>(a, s);
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "conv3x3 launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_conv3x3_wgrad(const void *x, const void *g, float *dw, float *dbias,
                                    int n_img, int H, int W, int c_in, int c_out, int accumulate,
                                    int *err, void *stream)
{
    if (!shape_ok(n_img, H, W, c_in, c_out))
        return set_global_error(LBM2P_EINVAL, "conv3x3_wgrad: need n_img, H, W >= 1 and C_in, C_out in {16, 32}");
    if (!x || !g || !dw || !err || !aligned16(x) || !aligned16(g))
        return set_global_error(LBM2P_EINVAL, "conv3x3_wgrad: x, g (16-byte aligned), dw and err are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!accumulate) {
        e = cudaMemsetAsync(dw, 0, (size_t)9 * c_in * c_out * sizeof(float), s);
        if (e == cudaSuccess && dbias)
            e = cudaMemsetAsync(dbias, 0, (size_t)c_out * sizeof(float), s);
        if (e != cudaSuccess)
            return set_global_error(LBM2P_ECUDA, "conv3x3_wgrad: clearing failed: %s", cudaGetErrorString(e));
    }
    WgradArgs a{};
    a.x = static_cast<const bf16 *>(x);
    a.g = static_cast<const bf16 *>(g);
    a.dw = dw;
    a.nimg = n_img;
    a.H = H;
    a.W = W;
    a.err = err;
    if (c_in == 16)
        e = c_out == 16 ? launch_wgrad<16, 16>(a, s) : launch_wgrad<16, 32>(a, s);
    else
        e = c_out == 16 ? launch_wgrad<32, 16>(a, s) : launch_wgrad<32, 32>(a, s);
    if (e == cudaSuccess && dbias) {
        const long long npix = (long long)n_img * H * W;
        k_bias_grad<<<grid_for(npix / 8 + 1, 1), 256, 0, s>>>(static_cast<const bf16 *>(g), dbias,
                                                               npix, c_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "conv3x3_wgrad launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_flip_weights(const void *w, void *wt, int c_in, int c_out, void *stream)
{
    if (!w || !wt || w == wt || !shape_ok(1, 1, 1, c_in, c_out))
        return set_global_error(LBM2P_EINVAL, "flip_weights: distinct w, wt and C_in, C_out in {16, 32}");
    const int n = 9 * c_in * c_out;
    k_flip<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(w), static_cast<bf16 *>(wt), c_in, c_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "flip_weights launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_adam(float *p, const float *g, float *m, float *v, void *pb, long long n,
                           float lr, float beta1, float beta2, float eps, int t, void *stream)
{
    if (!p || !g || !m || !v || n < 1 || t < 1 || !(lr > 0.0f) || !(eps > 0.0f) ||
        !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f))
        return set_global_error(LBM2P_EINVAL, "adam: bad arguments");
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_adam<<<grid_for(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        p, g, m, v, static_cast<bf16 *>(pb), n, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "adam launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_diff_stats(const float *a, const float *b, long long n, double *stats,
                                 void *stream)
{
    if (!a || !b || !stats || n < 1)
        return set_global_error(LBM2P_EINVAL, "diff_stats: bad arguments");
    k_diff_stats<<<grid_for(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a, b, n, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "diff_stats launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_features(const float *lnK, const float *S, const float *S_prev,
                               const float *P, const float *P_prev, const double *ds_stats,
                               const double *dp_stats, void *feat, int H, int W, float s_mean,
                               float s_scale, void *stream)
{
    if (!lnK || !S || !S_prev || !P || !P_prev || !ds_stats || !dp_stats || !feat || H < 1 ||
        W < 1 || !aligned16(feat) || !(s_scale > 0.0f))
        return set_global_error(LBM2P_EINVAL, "features: bad arguments");
    const long long n = (long long)H * W;
    k_features<<<grid_for(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        lnK, S, S_prev, P, P_prev, ds_stats, dp_stats, static_cast<bf16 *>(feat), n, s_mean,
        s_scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "features launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_target(const float *P_next, const float *P, const float *P_prev,
                             const double *dp_stats, float *tgt, int H, int W, void *stream)
{
    if (!P_next || !P || !P_prev || !dp_stats || !tgt || H < 1 || W < 1)
        return set_global_error(LBM2P_EINVAL, "target: bad arguments");
    const long long n = (long long)H * W;
    k_target<<<grid_for(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        P_next, P, P_prev, dp_stats, tgt, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "target launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_predict(const float *P, const float *P_prev, const float *d,
                              const double *dp_stats, float *P_pred, int H, int W, void *stream)
{
    if (!P || !P_prev || !d || !dp_stats || !P_pred || H < 1 || W < 1)
        return set_global_error(LBM2P_EINVAL, "predict: bad arguments");
    const long long n = (long long)H * W;
    k_predict<<<grid_for(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        P, P_prev, d, dp_stats, P_pred, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "predict launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

lbm2p_status lbm2p_op_mse_grad(const float *y0, const float *tgt, void *g, double *loss,
                               long long npix, int c_out, void *stream)
{
    if (!y0 || !tgt || !g || !loss || npix < 1 || (c_out != 16 && c_out != 32))
        return set_global_error(LBM2P_EINVAL, "mse_grad: bad arguments");
    k_mse_grad<<<grid_for(npix, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        y0, tgt, static_cast<bf16 *>(g), loss, npix, c_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "mse_grad launch failed: %s", cudaGetErrorString(e));
    return LBM2P_OK;
}

}  // extern "C"
