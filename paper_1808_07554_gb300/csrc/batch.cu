// Batched realisations: many independent lattices (handles made by lbm2p_create) advanced
// together.  One CUDA graph per physical step runs every member's saturation refresh,
// pressure sub-iteration and saturation update; each kernel walks one tile list that spans
// all members, so lattices too small to fill the GPU share it instead of each launching
// kernels that occupy a fraction of it.  The sub-iteration is a conditional WHILE node: a
// body runs check_every sweeps of every still-active member, then one block per member
// reduces that member's residual partials and retires it once its residual meets its
// tolerance (or its cap); the loop continues while any member is active.  Per node every
// kernel runs the device functions of the single-lattice kernels, so a member's state is
// bit-identical to stepping its handle alone with the same sweep counts.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "lbm2p.h"
#include "lbm2p_device.cuh"
#include "lbm2p_handle.h"
#include "lbm2p_node.cuh"

using namespace lbm2p_dev;

namespace {

// Device descriptor of one member: its kernel argument blocks for both f source parities
// and both step parities, and where its tiles sit in the batch tile list.  A tile is kBlock
// nodes: rpt rows of a (1 << wshift)-wide row segment, so lattices narrower than kBlock
// still fill the block.
struct Member {
    PressureArgs pa[2];          // sweep from the current f buffer A into B / from B into A
    RefreshArgs ra[2];           // batch step parity 0 / 1
    SaturationArgs sa[2];
    RebaseArgs rb;
    RebaseMidArgs rm;            // mid-solve rebase of the f buffer holding the state
    float *shift;                // the handle's residual conditioning constants
    long long nnodes;
    int nx, ny;
    int pf;                      // which of pa reads the buffer holding the state (0)
    int every;                   // sweeps between mid-solve rebases
    int wshift, rpt, seg_x;      // segment width 2^wshift, rows per tile, segments per row
    int tile0, ntiles;           // range in the batch tile list
    // A member of 512^2 nodes or more on a lattice with walls on every side ("pair" member)
    // is swept two sweeps per launch by k_pair_batch (blocks of 120 columns x h2 rows, nb2 of
    // them, residual partials at pb0 in the pair partials) instead of joining the one-sweep
    // batched sweep.  pparts / nparts: where finalize finds the member's residual partials
    // (the pair partials, or the batch's per-tile ones).
    int pair;                    // 1: a pair member
    int h2, nb2, pb0;
    const double *pparts;
    int nparts;
};

// per-member loop state of the current step
struct MemberCtl {
    int k;                       // sweeps run in this step
    int active;                  // still sub-iterating
    int cap;                     // sweep cap of this step
    int rebase;                  // move R to the current P before the next loop body
    double tol;                  // tolerance of this step (negative: run to the cap)
    double r;                    // last residual
};

__device__ __forceinline__ bool tile_node(const Member &M, int lt, int &x, int &y)
{
    const int ty = lt / M.seg_x;
    const int tx = lt - ty * M.seg_x;
    x = (tx << M.wshift) + (threadIdx.x & ((1 << M.wshift) - 1));
    y = ty * M.rpt + (threadIdx.x >> M.wshift);
    return x < M.nx && y < M.ny;
}

__global__ void __launch_bounds__(kBlock) kb_refresh(const Member *__restrict__ mem,
                                                     const int *__restrict__ tile_member,
                                                     int total, int q)
{
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const Member &M = mem[tile_member[t]];
        int x, y;
        if (tile_node(M, t - M.tile0, x, y))
            refresh_node(M.ra[q], x, y, y * M.ra[q].g.pitch + x);
    }
}

__global__ void kb_reset(MemberCtl *ctl, const int *__restrict__ caps,
                         const double *__restrict__ tols, int count, int *active_count)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m == 0)
        active_count[0] = active_count[1] = 0;
    if (m < count) {
        ctl[m].k = 0;
        ctl[m].cap = caps[m];
        ctl[m].tol = tols[m];
        ctl[m].active = caps[m] > 0 ? 1 : 0;
        ctl[m].rebase = 0;
        ctl[m].r = nan("");
    }
}

// Sweep number idx (0-based) of a loop body over the tiles of the still-active members:
// act[0 .. counts[2]) lists (member, tile of the member), rebuilt after every body.
template <bool CHECK, bool WRITE_P>
__global__ void __launch_bounds__(kBlock) kb_sweep(const Member *__restrict__ mem,
                                                   const int2 *__restrict__ act,
                                                   const int *__restrict__ counts, int idx,
                                                   double *__restrict__ partials)
{
    __shared__ double red[kBlock / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = counts[2];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int2 e = act[t];
        const Member &M = mem[e.x];
        const PressureArgs &a = M.pa[M.pf ^ (idx & 1)];
        float d = 0.0f, q = 0.0f;
        int x, y;
        const float shift = CHECK ? M.shift[0] : 0.0f;
        const float dshift = CHECK ? M.shift[1] : 0.0f;
        if (tile_node(M, e.y, x, y))
            sweep_node<CHECK, WRITE_P>(a, x, y, y * a.g.pitch + x, shift, dshift, d, q);
        if (CHECK) {
            const float s0 = warp_sum(d), s1 = warp_sum(d * d), s2 = warp_sum(q), s3 = warp_sum(q * q);
            if (lane == 0) {
                red[warp][0] = s0;
                red[warp][1] = s1;
                red[warp][2] = s2;
                red[warp][3] = s3;
            }
            __syncthreads();
            if (threadIdx.x < 4) {
                double s = 0.0;
#pragma unroll
                for (int w = 0; w < kBlock / 32; ++w)
                    s += red[w][threadIdx.x];
                partials[4 * (size_t)(M.tile0 + e.y) + threadIdx.x] = s;
            }
            __syncthreads();
        }
    }
}

// One block per member: the residual of its last sweep (the stopping test of Sec. 3, with
// the arithmetic of the single-lattice finalize), then retire it or keep it active, and
// mark it for a mid-solve rebase on the rule of the single-lattice loop.  counts[0] counts
// the members still active, counts[1] those to rebase.
__global__ void __launch_bounds__(256) kb_finalize(const Member *__restrict__ mem,
                                                   const double *__restrict__ partials,
                                                   MemberCtl *ctl, int body, int *counts)
{
    const int mi = blockIdx.x;
    MemberCtl &c = ctl[mi];
    if (!c.active)
        return;                                         // uniform over the block
    const Member &M = mem[mi];
    __shared__ double red[256][4];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    (void)partials;
    for (int i = threadIdx.x; i < M.nparts; i += 256)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            s[q] += M.pparts[4 * (size_t)i + q];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        red[threadIdx.x][q] = s[q];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                red[threadIdx.x][q] += red[threadIdx.x + h][q];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double N = (double)M.nnodes;
        const double sd = red[0][0], sdd = red[0][1], sp = red[0][2], spp = red[0][3];
        const double c0 = (double)M.shift[0], c1 = (double)M.shift[1];
        double r;
        if (!isfinite(sd) || !isfinite(sdd) || !isfinite(sp) || !isfinite(spp)) {
            r = nan("");
        } else {
            double num = sdd - sd * sd / N, den = spp - sp * sp / N;
            num = num > 0.0 ? num : 0.0;
            den = den > 0.0 ? den : 0.0;
            r = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
            M.shift[0] = (float)(c0 + sp / N);
            M.shift[1] = (float)(c1 + sd / N);
        }
        c.k += body;
        c.r = r;
        const bool more = !(r <= c.tol) && !isnan(r) && c.k < c.cap;
        const bool rebase = more && M.every > 0 && c.k % M.every == 0;
        c.active = more ? 1 : 0;
        c.rebase = rebase ? 1 : 0;
        if (more)
            atomicAdd(&counts[0], 1);
        if (rebase)
            atomicAdd(&counts[1], 1);
    }
}

// One block: (SET) continue the loop while a member is active and rebase when one asks;
// then the exclusive prefix of the active members' tile counts, counts[2] = their total.
template <bool SET>
__global__ void __launch_bounds__(256) kb_prefix(const Member *__restrict__ mem,
                                                 const MemberCtl *__restrict__ ctl, int count,
                                                 int *__restrict__ prefix, int *counts,
                                                 cudaGraphConditionalHandle h_loop,
                                                 cudaGraphConditionalHandle h_rebase)
{
    __shared__ int scan[2][256];
    __shared__ int carry[2];
    if (threadIdx.x == 0) {
        if (SET) {
            const int active = counts[0], rebase = counts[1];
            counts[0] = counts[1] = 0;
            cudaGraphSetConditional(h_loop, active > 0 ? 1u : 0u);
            cudaGraphSetConditional(h_rebase, rebase > 0 ? 1u : 0u);
        }
        carry[0] = carry[1] = 0;
    }
    __syncthreads();
    // two exclusive prefixes at once: tiles of the one-sweep members, blocks of the pair
    // members (a member is one or the other, so one prefix array holds both)
    for (int base = 0; base < count; base += 256) {
        const int m = base + (int)threadIdx.x;
        const bool on = m < count && ctl[m].active;
        const int pair = on && mem[m].pair;
        const int v = on ? (pair ? mem[m].nb2 : mem[m].ntiles) : 0;
        scan[0][threadIdx.x] = pair ? 0 : v;
        scan[1][threadIdx.x] = pair ? v : 0;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {        // inclusive scans
            const int a0 = (int)threadIdx.x >= off ? scan[0][threadIdx.x - off] : 0;
            const int a1 = (int)threadIdx.x >= off ? scan[1][threadIdx.x - off] : 0;
            __syncthreads();
            scan[0][threadIdx.x] += a0;
            scan[1][threadIdx.x] += a1;
            __syncthreads();
        }
        if (m < count)
            prefix[m] = carry[pair] + scan[pair][threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 255) {
            carry[0] += scan[0][255];
            carry[1] += scan[1][255];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts[2] = carry[0];
        counts[3] = carry[1];
    }
}

// one block per member: list the tiles of an active one-sweep member (act) or the blocks of an
// active pair member (items) at its prefix offset
__global__ void __launch_bounds__(256) kb_scatter(const Member *__restrict__ mem,
                                                  const MemberCtl *__restrict__ ctl,
                                                  const int *__restrict__ prefix,
                                                  int2 *__restrict__ act, int2 *__restrict__ items)
{
    const int m = blockIdx.x;
    if (!ctl[m].active)
        return;
    const bool pair = mem[m].pair != 0;
    const int base = prefix[m], n = pair ? mem[m].nb2 : mem[m].ntiles;
    int2 *dst = pair ? items : act;
    for (int i = threadIdx.x; i < n; i += 256)
        dst[base + i] = make_int2(m, i);
}

__global__ void __launch_bounds__(kBlock) kb_rebase_mid(const Member *__restrict__ mem,
                                                        const int *__restrict__ tile_member,
                                                        int total, const MemberCtl *__restrict__ ctl)
{
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int mi = tile_member[t];
        if (!ctl[mi].rebase)
            continue;
        const Member &M = mem[mi];
        int x, y;
        if (tile_node(M, t - M.tile0, x, y))
            rebase_mid_node(M.rm, y * M.rm.g.pitch + x);
    }
}

__global__ void __launch_bounds__(kBlock) kb_saturation(const Member *__restrict__ mem,
                                                        const int *__restrict__ tile_member,
                                                        int total, int q)
{
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const Member &M = mem[tile_member[t]];
        int x, y;
        if (tile_node(M, t - M.tile0, x, y))
            saturation_node(M.sa[q], x, y, y * M.sa[q].g.pitch + x);
    }
}

__global__ void __launch_bounds__(kBlock) kb_rebase(const Member *__restrict__ mem,
                                                    const int *__restrict__ tile_member, int total)
{
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const Member &M = mem[tile_member[t]];
        int x, y;
        if (tile_node(M, t - M.tile0, x, y))
            rebase_node(M.rb, y * M.rb.g.pitch + x);
    }
}

}  // namespace

struct lbm2p_batch {
    std::vector<lbm2p *> members;
    std::vector<int> pf, pg0, pr;        // member buffers the graphs were built for
    int count = 0, total = 0, body = 0, grid = 0, grid_check = 0;
    void *stream = nullptr;
    Member *d_mem = nullptr;
    int *d_tile_member = nullptr;
    MemberCtl *d_ctl = nullptr;
    MemberCtl *h_ctl = nullptr;          // pinned
    int *d_caps = nullptr;
    double *d_tols = nullptr;
    int *h_caps = nullptr;               // pinned
    double *h_tols = nullptr;            // pinned
    int *d_active = nullptr;             // [0] active members, [1] members to rebase,
                                         // [2] tiles of the active one-sweep members,
                                         // [3] blocks of the active pair members
    int *d_prefix = nullptr;             // first compacted tile (block) of each active member
    int2 *d_act = nullptr;               // compacted (member, tile) list
    double *d_partials = nullptr;
    int npair = 0, pair_total = 0;       // pair members, their blocks
    int pair_grid = 0;                   // blocks of a k_pair_batch launch
    PressureArgs *d_pa2 = nullptr;       // [2 count] argument blocks of the pair launches
    int *d_h2 = nullptr, *d_pb0 = nullptr;   // [count] block height, first partial
    int2 *d_items = nullptr;             // compacted (member, block) list of the pair members
    double *d_pparts = nullptr;          // [4 pair_total] their residual partials
    cudaGraph_t graph[2] = {};
    cudaGraphExec_t exec[2] = {};
    int gstep = 0;                       // parity of the steps run by the batch
    long long launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
};

namespace {

lbm2p_status bfail(lbm2p_batch *b, lbm2p_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b)
        b->err = buf;
    lbm2p_internal::set_global_error(st, "%s", buf);
    return st;
}

#define BTRY(b, call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return bfail((b), LBM2P_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

void batch_free(lbm2p_batch *b)
{
    for (int q = 0; q < 2; ++q) {
        if (b->exec[q])
            cudaGraphExecDestroy(b->exec[q]);
        if (b->graph[q])
            cudaGraphDestroy(b->graph[q]);
    }
    cudaFree(b->d_mem);
    cudaFree(b->d_tile_member);
    cudaFree(b->d_ctl);
    cudaFree(b->d_caps);
    cudaFree(b->d_tols);
    cudaFree(b->d_active);
    cudaFree(b->d_prefix);
    cudaFree(b->d_act);
    cudaFree(b->d_pa2);
    cudaFree(b->d_h2);
    cudaFree(b->d_pb0);
    cudaFree(b->d_items);
    cudaFree(b->d_pparts);
    cudaFree(b->d_partials);
    if (b->h_ctl)
        cudaFreeHost(b->h_ctl);
    if (b->h_caps)
        cudaFreeHost(b->h_caps);
    if (b->h_tols)
        cudaFreeHost(b->h_tols);
    if (b->ev0)
        cudaEventDestroy(b->ev0);
    if (b->ev1)
        cudaEventDestroy(b->ev1);
}

cudaError_t add_k(cudaGraphNode_t *n, cudaGraph_t g, const cudaGraphNode_t *dep, void *func,
                  int grid, int block, void **args)
{
    cudaKernelNodeParams p{};
    p.func = func;
    p.gridDim = dim3((unsigned)grid);
    p.blockDim = dim3((unsigned)block);
    p.kernelParams = args;
    return cudaGraphAddKernelNode(n, g, dep, dep ? 1 : 0, &p);
}

void *sweep_kernel(bool check, bool write_p)
{
    return check ? (write_p ? (void *)kb_sweep<true, true> : (void *)kb_sweep<true, false>)
                 : (write_p ? (void *)kb_sweep<false, true> : (void *)kb_sweep<false, false>);
}

// the graph of one batched step at step parity q (the g buffers swap every step):
// refresh -> reset -> prefix -> scatter -> WHILE{ body sweeps -> finalize -> condition +
// prefix -> scatter -> IF{ mid-solve rebase } } -> saturation -> rebase
lbm2p_status build_graph(lbm2p_batch *b, int q)
{
    cudaGraph_t G;
    BTRY(b, cudaGraphCreate(&G, 0));
    b->graph[q] = G;
    const Member *mem = b->d_mem;
    const int *tm = b->d_tile_member;
    int count = b->count, total = b->total;
    MemberCtl *ctl = b->d_ctl;
    const MemberCtl *cctl = b->d_ctl;
    const int *caps = b->d_caps;
    const double *tols = b->d_tols;
    int *act = b->d_active;
    double *partials = b->d_partials;
    const double *cpartials = b->d_partials;
    int *prefix = b->d_prefix;
    const int *cprefix = b->d_prefix;
    int2 *actl = b->d_act;
    const int2 *cactl = b->d_act;
    const int *cact = b->d_active;
    int body = b->body;
    cudaGraphNode_t nr, nreset, npre, nsc, nw, nsat, nreb;
    {
        void *args[] = {(void *)&mem, (void *)&tm, (void *)&total, (void *)&q};
        BTRY(b, add_k(&nr, G, nullptr, (void *)kb_refresh, b->grid, kBlock, args));
    }
    {
        void *args[] = {(void *)&ctl, (void *)&caps, (void *)&tols, (void *)&count, (void *)&act};
        BTRY(b, add_k(&nreset, G, &nr, (void *)kb_reset, (count + 255) / 256, 256, args));
    }
    cudaGraphConditionalHandle hd, hnone{};
    BTRY(b, cudaGraphConditionalHandleCreate(&hd, G, 1, cudaGraphCondAssignDefault));
    int2 *items = b->d_items;
    {
        void *args[] = {(void *)&mem, (void *)&cctl, (void *)&count, (void *)&prefix,
                        (void *)&act, (void *)&hnone, (void *)&hnone};
        BTRY(b, add_k(&npre, G, &nreset, (void *)kb_prefix<false>, 1, 256, args));
    }
    {
        void *args[] = {(void *)&mem, (void *)&cctl, (void *)&cprefix, (void *)&actl,
                        (void *)&items};
        BTRY(b, add_k(&nsc, G, &npre, (void *)kb_scatter, count, 256, args));
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    BTRY(b, cudaGraphAddNode(&nw, G, &nsc, nullptr, 1, &cp));
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    for (int kk = 0; kk < body; ++kk) {
        const bool check = kk == body - 1, write_p = kk == body - 2;
        int idx = kk;
        void *args[] = {(void *)&mem, (void *)&cactl, (void *)&cact, (void *)&idx,
                        (void *)&partials};
        cudaGraphNode_t n;
        BTRY(b, add_k(&n, bg, prev ? &prev : nullptr, sweep_kernel(check, write_p),
                      check ? b->grid_check : b->grid, kBlock, args));
        prev = n;
    }
    // the pair members: check_every / 2 launches of k_pair_batch (two sweeps each, over the
    // blocks of every pair member still iterating), a chain beside the one-sweep chain
    std::vector<cudaGraphNode_t> ends{prev};
    if (b->npair > 0) {
        cudaGraphNode_t p2 = nullptr;
        for (int kk = 0; kk < body / 2; ++kk) {
            cudaGraphNode_t n;
            BTRY(b, lbm2p_launch::node_pair_batch(&n, bg, p2 ? &p2 : nullptr, b->d_pa2, b->d_h2,
                                                  b->d_pb0, b->d_items, b->d_active + 3, kk & 1,
                                                  kk == body / 2 - 1, b->d_pparts, b->pair_grid));
            p2 = n;
        }
        ends.push_back(p2);
    }
    cudaGraphNode_t nf, nc, nsc2, nif, nrm;
    {
        void *args[] = {(void *)&mem, (void *)&cpartials, (void *)&ctl, (void *)&body, (void *)&act};
        cudaKernelNodeParams kp{};
        kp.func = (void *)kb_finalize;
        kp.gridDim = dim3((unsigned)count);
        kp.blockDim = dim3(256u);
        kp.kernelParams = args;
        BTRY(b, cudaGraphAddKernelNode(&nf, bg, ends.data(), ends.size(), &kp));
    }
    cudaGraphConditionalHandle hr;
    BTRY(b, cudaGraphConditionalHandleCreate(&hr, bg, 0, 0));
    {
        void *args[] = {(void *)&mem, (void *)&cctl, (void *)&count, (void *)&prefix,
                        (void *)&act, (void *)&hd, (void *)&hr};
        BTRY(b, add_k(&nc, bg, &nf, (void *)kb_prefix<true>, 1, 256, args));
    }
    {
        void *args[] = {(void *)&mem, (void *)&cctl, (void *)&cprefix, (void *)&actl,
                        (void *)&items};
        BTRY(b, add_k(&nsc2, bg, &nc, (void *)kb_scatter, count, 256, args));
    }
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hr;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    BTRY(b, cudaGraphAddNode(&nif, bg, &nsc2, nullptr, 1, &ip));
    {
        void *args[] = {(void *)&mem, (void *)&tm, (void *)&total, (void *)&cctl};
        BTRY(b, add_k(&nrm, ip.conditional.phGraph_out[0], nullptr, (void *)kb_rebase_mid,
                      b->grid, kBlock, args));
    }
    {
        void *args[] = {(void *)&mem, (void *)&tm, (void *)&total, (void *)&q};
        BTRY(b, add_k(&nsat, G, &nw, (void *)kb_saturation, b->grid, kBlock, args));
    }
    {
        void *args[] = {(void *)&mem, (void *)&tm, (void *)&total};
        BTRY(b, add_k(&nreb, G, &nsat, (void *)kb_rebase, b->grid, kBlock, args));
    }
    BTRY(b, cudaGraphInstantiate(&b->exec[q], G, 0));
    return LBM2P_OK;
}

}  // namespace

extern "C" {

lbm2p_status lbm2p_batch_create(lbm2p_batch **out, lbm2p *const *members, int count)
{
    if (!out)
        return bfail(nullptr, LBM2P_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (!members || count < 1)
        return bfail(nullptr, LBM2P_EINVAL, "a batch needs at least one member");
    const lbm2p *m0 = members[0];
    if (!m0)
        return bfail(nullptr, LBM2P_EINVAL, "member 0 is NULL");
    for (int i = 0; i < count; ++i) {
        const lbm2p *h = members[i];
        if (!h)
            return bfail(nullptr, LBM2P_EINVAL, "member %d is NULL", i);
        if (h->stream != m0->stream)
            return bfail(nullptr, LBM2P_EINVAL, "member %d uses another stream than member 0", i);
        if (h->p.check_every != m0->p.check_every || h->p.check_every < 2 || h->p.check_every % 2)
            return bfail(nullptr, LBM2P_EINVAL,
                         "members need one even check_every (member %d has %d, member 0 %d)", i,
                         h->p.check_every, m0->p.check_every);
        if (h->fp16)
            return bfail(nullptr, LBM2P_EINVAL, "member %d uses FP16 storage (not batched)", i);
        if (h->p.max_sub_iters % h->p.check_every)
            return bfail(nullptr, LBM2P_EINVAL,
                         "member %d: max_sub_iters %d is not a multiple of check_every %d", i,
                         h->p.max_sub_iters, h->p.check_every);
        for (int j = 0; j < i; ++j)
            if (members[j] == h)
                return bfail(nullptr, LBM2P_EINVAL, "member %d appears twice", i);
    }
    lbm2p_batch *b = new (std::nothrow) lbm2p_batch();
    if (!b)
        return bfail(nullptr, LBM2P_ENOMEM, "host allocation failed");
    b->members.assign(members, members + count);
    b->count = count;
    b->body = m0->p.check_every;
    b->stream = m0->stream;
    std::vector<Member> hm((size_t)count);
    std::vector<PressureArgs> pa2(2 * (size_t)count);
    std::vector<int> h2v((size_t)count), pb0v((size_t)count);
    std::vector<int> tile_member;
    int total = 0;
    for (int i = 0; i < count; ++i) {
        lbm2p *h = members[i];
        Member &M = hm[(size_t)i];
        // the batch ping-pongs each member between its current f buffer A and the next one
        // of the rotation, B (a loop body is an even number of sweeps, so a step ends in A),
        // and updates R, 1/tau_f and P^{n-1} in place
        const int A = h->cur_f, B = lbm2p_internal::fnext(A, 1);
        M.pa[0] = lbm2p_internal::pressure_args(h, A, B, false);
        M.pa[1] = lbm2p_internal::pressure_args(h, B, A, false);
        for (int q = 0; q < 2; ++q) {
            M.pa[q].partials = nullptr;
            M.ra[q] = lbm2p_internal::refresh_args(h, h->cur_g ^ q, true);
            M.sa[q] = lbm2p_internal::saturation_args(h, A, h->cur_g ^ q, false);
        }
        M.rb = lbm2p_internal::rebase_args(h, A, false);
        M.rm = lbm2p_internal::rebase_mid_args(h, A, false);
        M.every = h->rebase_every;
        M.shift = h->shift;
        M.nnodes = h->nnodes;
        M.nx = h->nx;
        M.ny = h->ny;
        M.pf = 0;                      // pa[0] reads A
        int w = 32;
        while (w < h->nx && w < kBlock)
            w *= 2;
        M.wshift = 0;
        while ((1 << M.wshift) < w)
            ++M.wshift;
        M.rpt = kBlock / w;
        M.seg_x = (h->nx + w - 1) / w;
        M.tile0 = total;
        M.ntiles = M.seg_x * ((h->ny + M.rpt - 1) / M.rpt);
        total += M.ntiles;
        tile_member.insert(tile_member.end(), (size_t)M.ntiles, i);
        // members of 512^2 nodes and more with walls on every side sweep two at a time
        // (k_pair_batch; a body of check_every sweeps is then check_every / 2 launches, an
        // even number, ending in buffer A), in blocks of the height their handle's tuning
        // chose for the direct-load form, else 4 rows
        bool walls = true;
        for (int sd = 0; sd < 4; ++sd)
            walls = walls && h->p.bc[sd] != LBM2P_BC_PERIODIC;
        M.pair = (!h->fp16 && walls && h->nnodes >= 512LL * 512 && b->body % 4 == 0) ? 1 : 0;
        M.h2 = M.nb2 = M.pb0 = 0;
        if (M.pair) {
            M.h2 = (h->tb_T > 1 && h->tb_kind == 2 && h->tb_W == 120) ? h->tb_H : 4;
            M.h2 = M.h2 < h->ny ? M.h2 : h->ny;
            M.nb2 = (int)lbm2p_launch::pair_direct_grid(4, M.h2, h->nx, h->ny);
            M.pb0 = b->pair_total;
            b->pair_total += M.nb2;
            ++b->npair;
        }
        pa2[2 * (size_t)i] = M.pa[0];
        pa2[2 * (size_t)i + 1] = M.pa[1];
        h2v[(size_t)i] = M.h2;
        pb0v[(size_t)i] = M.pb0;
        M.pparts = nullptr;                    // set once the partials are allocated
        M.nparts = M.pair ? M.nb2 : M.ntiles;
        b->pf.push_back(h->cur_f);
        b->pg0.push_back(h->cur_g);
        b->pr.push_back(h->cur_r);
    }
    b->total = total;
    int dev = 0, sms = 0, per = 0, perc = 0;
    lbm2p_status st = LBM2P_OK;
    auto ok = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == LBM2P_OK)
            st = bfail(b, e == cudaErrorMemoryAllocation ? LBM2P_ENOMEM : LBM2P_ECUDA,
                       "%s failed: %s", what, cudaGetErrorString(e));
        return st == LBM2P_OK;
    };
    ok(cudaGetDevice(&dev), "cudaGetDevice") &&
        ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute") &&
        ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kb_sweep<false, true>, kBlock, 0),
           "cudaOccupancyMaxActiveBlocksPerMultiprocessor") &&
        ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perc, kb_sweep<true, false>, kBlock, 0),
           "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (st == LBM2P_OK) {
        const long long g1 = (long long)sms * (per > 0 ? per : 1);
        const long long g2 = (long long)sms * (perc > 0 ? perc : 1);
        b->grid = (int)(g1 < total ? g1 : total);
        b->grid_check = (int)(g2 < total ? g2 : total);
        const long long g3 = (long long)sms * lbm2p_launch::pair_batch_blocks_per_sm();
        b->pair_grid = (int)(g3 < b->pair_total ? g3 : (b->pair_total > 0 ? b->pair_total : 1));
        ok(cudaMalloc(&b->d_mem, sizeof(Member) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_tile_member, sizeof(int) * (size_t)total), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_ctl, sizeof(MemberCtl) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_caps, sizeof(int) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_tols, sizeof(double) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_active, 4 * sizeof(int)), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_prefix, sizeof(int) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_act, sizeof(int2) * (size_t)total), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_partials, sizeof(double) * 4 * (size_t)total), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_pa2, sizeof(PressureArgs) * 2 * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_h2, sizeof(int) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_pb0, sizeof(int) * (size_t)count), "cudaMalloc") &&
            ok(cudaMalloc(&b->d_items, sizeof(int2) * (size_t)(b->pair_total > 0 ? b->pair_total : 1)),
               "cudaMalloc") &&
            ok(cudaMalloc(&b->d_pparts,
                          sizeof(double) * 4 * (size_t)(b->pair_total > 0 ? b->pair_total : 1)),
               "cudaMalloc") &&
            ok(cudaMallocHost(&b->h_ctl, sizeof(MemberCtl) * (size_t)count), "cudaMallocHost") &&
            ok(cudaMallocHost(&b->h_caps, sizeof(int) * (size_t)count), "cudaMallocHost") &&
            ok(cudaMallocHost(&b->h_tols, sizeof(double) * (size_t)count), "cudaMallocHost") &&
            ok(cudaEventCreate(&b->ev0), "cudaEventCreate") &&
            ok(cudaEventCreate(&b->ev1), "cudaEventCreate");
    }
    if (st == LBM2P_OK) {
        // residual partials: one per tile of each one-sweep member, one per block of each
        // pair member
        for (int i = 0; i < count; ++i) {
            Member &M = hm[(size_t)i];
            M.pparts = M.pair ? b->d_pparts + 4 * (size_t)M.pb0 : b->d_partials + 4 * (size_t)M.tile0;
        }
        cudaStream_t cs = (cudaStream_t)b->stream;
        ok(cudaMemcpyAsync(b->d_mem, hm.data(), sizeof(Member) * (size_t)count,
                           cudaMemcpyHostToDevice, cs), "cudaMemcpyAsync") &&
            ok(cudaMemcpyAsync(b->d_pa2, pa2.data(), sizeof(PressureArgs) * 2 * (size_t)count,
                               cudaMemcpyHostToDevice, cs), "cudaMemcpyAsync") &&
            ok(cudaMemcpyAsync(b->d_h2, h2v.data(), sizeof(int) * (size_t)count,
                               cudaMemcpyHostToDevice, cs), "cudaMemcpyAsync") &&
            ok(cudaMemcpyAsync(b->d_pb0, pb0v.data(), sizeof(int) * (size_t)count,
                               cudaMemcpyHostToDevice, cs), "cudaMemcpyAsync") &&
            ok(cudaMemcpyAsync(b->d_tile_member, tile_member.data(), sizeof(int) * (size_t)total,
                               cudaMemcpyHostToDevice, cs), "cudaMemcpyAsync") &&
            ok(cudaMemsetAsync(b->d_ctl, 0, sizeof(MemberCtl) * (size_t)count, cs), "cudaMemsetAsync") &&
            ok(cudaMemsetAsync(b->d_active, 0, 4 * sizeof(int), cs), "cudaMemsetAsync") &&
            ok(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
    }
    for (int q = 0; q < 2 && st == LBM2P_OK; ++q)
        st = build_graph(b, q);
    if (st != LBM2P_OK) {
        batch_free(b);
        delete b;
        return st;
    }
    *out = b;
    return LBM2P_OK;
}

lbm2p_status lbm2p_batch_step(lbm2p_batch *b, int nsteps, const int *replay,
                              lbm2p_step_stats *stats)
{
    if (!b)
        return bfail(nullptr, LBM2P_EINVAL, "NULL batch");
    if (nsteps < 0)
        return bfail(b, LBM2P_EINVAL, "nsteps must be >= 0");
    if (replay)
        for (long long i = 0; i < (long long)nsteps * b->count; ++i)
            if (replay[i] < 0 || replay[i] % b->body)
                return bfail(b, LBM2P_EINVAL,
                             "replay counts must be non-negative multiples of %d (entry %lld is %d)",
                             b->body, i, replay[i]);
    for (int m = 0; m < b->count; ++m) {
        const lbm2p *h = b->members[(size_t)m];
        if (h->cur_f != b->pf[(size_t)m] || h->cur_r != b->pr[(size_t)m] ||
            h->cur_g != (b->pg0[(size_t)m] ^ b->gstep))
            return bfail(b, LBM2P_EINVAL,
                         "member %d was stepped outside the batch (buffer parity changed)", m);
    }
    cudaStream_t cs = (cudaStream_t)b->stream;
    lbm2p_status worst = LBM2P_OK;
    for (int s = 0; s < nsteps; ++s) {
        for (int m = 0; m < b->count; ++m) {
            const lbm2p *h = b->members[(size_t)m];
            if (replay) {
                b->h_caps[m] = replay[(size_t)s * b->count + m];
                b->h_tols[m] = -1.0;
            } else {
                b->h_caps[m] = h->p.max_sub_iters;
                b->h_tols[m] = h->p.tol;
            }
        }
        BTRY(b, cudaMemcpyAsync(b->d_caps, b->h_caps, sizeof(int) * (size_t)b->count,
                                cudaMemcpyHostToDevice, cs));
        BTRY(b, cudaMemcpyAsync(b->d_tols, b->h_tols, sizeof(double) * (size_t)b->count,
                                cudaMemcpyHostToDevice, cs));
        BTRY(b, cudaEventRecord(b->ev0, cs));
        BTRY(b, cudaGraphLaunch(b->exec[b->gstep], cs));
        BTRY(b, cudaEventRecord(b->ev1, cs));
        BTRY(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(MemberCtl) * (size_t)b->count,
                                cudaMemcpyDeviceToHost, cs));
        BTRY(b, cudaStreamSynchronize(cs));
        float ms = -1.0f;
        BTRY(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        b->gstep ^= 1;
        int kmax = 0;
        for (int m = 0; m < b->count; ++m) {
            lbm2p *h = b->members[(size_t)m];
            const MemberCtl &c = b->h_ctl[m];
            h->cur_g = 1 - h->cur_g;
            h->sweeps += c.k;
            kmax = c.k > kmax ? c.k : kmax;
            lbm2p_status mst = LBM2P_OK;
            if (c.k > 0 && std::isnan(c.r))
                mst = LBM2P_ENONFINITE;
            else if (!replay && !(c.r <= h->p.tol))
                mst = LBM2P_ENOTCONVERGED;
            if (mst == LBM2P_ENONFINITE || (mst != LBM2P_OK && worst == LBM2P_OK))
                worst = mst;
            if (stats) {
                lbm2p_step_stats &o = stats[(size_t)s * b->count + m];
                o.sub_iters = c.k;
                o.status = mst;
                o.residual = c.r;
                o.sweep_ms = -1.0f;
                o.step_ms = ms;
            }
        }
        // refresh, reset, prefix, scatter, saturation, rebase; per loop pass: body sweeps,
        // finalize, condition + prefix, scatter; and the mid-solve rebases of the longest solve
        const int passes = kmax > 0 ? kmax / b->body : 1;
        const int every = b->body * ((1024 + b->body - 1) / b->body);
        b->launches += 6 + (long long)passes * (b->body + 3) + (kmax > 0 ? (kmax - 1) / every : 0);
        if (b->npair > 0)                      // the pair members' body / 2 launches a pass
            b->launches += (long long)passes * (b->body / 2);
        if (worst == LBM2P_ENONFINITE)
            return bfail(b, worst, "a member's pressure residual is not finite (step %d)", s);
    }
    if (worst == LBM2P_ENOTCONVERGED)
        bfail(b, worst, "a member reached its sweep cap before its tolerance");
    return worst;
}

lbm2p_status lbm2p_batch_counters(const lbm2p_batch *b, long long *launches, int *total_tiles)
{
    if (!b)
        return bfail(nullptr, LBM2P_EINVAL, "NULL batch");
    if (launches)
        *launches = b->launches;
    if (total_tiles)
        *total_tiles = b->total;
    return LBM2P_OK;
}

const char *lbm2p_batch_last_error(const lbm2p_batch *b)
{
    return b ? b->err.c_str() : lbm2p_last_error(nullptr);
}

void lbm2p_batch_destroy(lbm2p_batch *b)
{
    if (!b)
        return;
    cudaStreamSynchronize((cudaStream_t)b->stream);
    batch_free(b);
    delete b;
}

}  // extern "C"
