// lbm2p_pressure_sweep_noalloc: one pressure sweep with its residual, for callers that
// cannot allocate device memory.
//
// Some host programs must not call cudaMalloc at run time: codes that hand every byte of
// device memory to their own pool at start-up, real-time loops that forbid allocation
// after initialisation, and plug-ins running inside a host application that owns the
// device allocator.  They can still run the solver's hot kernel on buffers they already
// own.  The only device memory the sweep needs beyond its inputs and outputs is the
// scratch of the residual reduction (four FP64 partials per row tile, the finalize output
// and two shifts), and here that scratch is a file-scope static device array: it is part of
// the loaded library image, present on every GPU that loads the library until the process
// exits, and no call of this entry point allocates or frees anything.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "lbm2p.h"
#include "lbm2p_device.cuh"

using namespace lbm2p_dev;

namespace {

// Layout of the scratch array (doubles): [0, 4 * MAX_TILES) residual partials, 4 per row
// tile; then the finalize output (ResidualOut); then the shift (a float in one slot).
constexpr size_t kPartials = 4 * (size_t)LBM2P_NOALLOC_MAX_TILES;
constexpr size_t kOutSlots = (sizeof(ResidualOut) + sizeof(double) - 1) / sizeof(double);
constexpr size_t kScratchDoubles = kPartials + kOutSlots + 1;   // last slot: two float shifts

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// cached device address of the scratch array, per device, valid for the CUDA context whose
// unique id is stored beside it (a context id is never reused within a process)
double *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// driver calls reached through the runtime (no link against the driver library)
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);

// Unique id of the current device's context.  A cudaDeviceReset destroys the primary context
// and the next call creates a new one, with the library's module loaded anew (the array can
// move), and a new id.
lbm2p_status current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                          cudaEnableDefault, &q1);
        cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                          cudaEnableDefault, &q2);
        if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return lbm2p_internal::set_global_error(LBM2P_ECUDA,
                                                    "the driver's context queries are unavailable");
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0)
        return lbm2p_internal::set_global_error(LBM2P_ECUDA, "no current CUDA context");
    return LBM2P_OK;
}

// Device address of the scratch array on the current device.  The host-side name of the
// array is only a stand-in, so the address is looked up with that device current, once per
// device and context (the first call after a context is created), and cached.
lbm2p_status scratch_on_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaSetDevice(dev);         // makes the device's primary context current
    if (e != cudaSuccess)
        return lbm2p_internal::set_global_error(LBM2P_ECUDA, "no usable CUDA device: %s",
                                                cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return lbm2p_internal::set_global_error(LBM2P_EINVAL, "device ordinal %d above %d", dev,
                                                kMaxDevices - 1);
    unsigned long long ctx = 0;
    lbm2p_status st = current_context_id(&ctx);
    if (st != LBM2P_OK)
        return st;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return lbm2p_internal::set_global_error(LBM2P_ECUDA,
                                                    "cudaGetSymbolAddress of the sweep scratch "
                                                    "failed on device %d: %s",
                                                    dev, cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return LBM2P_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" lbm2p_status lbm2p_pressure_sweep_noalloc(int nx, int ny, int pitch, const int bc[4],
                                                     const float *const n_in[8],
                                                     float *const n_out[8], const float *R,
                                                     const float *inv_tau, const float *Fp,
                                                     const float *const P_b[4], float *dP,
                                                     double *residual, void *stream)
{
    using lbm2p_internal::set_global_error;
    if (nx < 1 || ny < 1 || pitch < nx || pitch % 4 != 0)
        return set_global_error(LBM2P_EINVAL, "need nx, ny >= 1 and pitch >= nx, a multiple of 4");
    if ((long long)pitch * ny >= (1LL << 31) - 1024)
        return set_global_error(LBM2P_EINVAL, "lattice %d x %d exceeds the 2^31 plane limit", nx, ny);
    const long long tiles_x = (nx + 4LL * kBlock - 1) / (4LL * kBlock);
    const long long tiles = tiles_x * ny;
    if (tiles > LBM2P_NOALLOC_MAX_TILES)
        return set_global_error(LBM2P_EINVAL,
                                "lattice %d x %d has %lld row tiles of %d nodes; the static "
                                "scratch holds %d (use the handle-based lbm2p_step)",
                                nx, ny, tiles, 4 * kBlock, LBM2P_NOALLOC_MAX_TILES);
    if (!bc || !n_in || !n_out || !R || !inv_tau || !dP || !residual)
        return set_global_error(LBM2P_EINVAL, "bc, n_in, n_out, R, inv_tau, dP and residual are required");
    for (int s = 0; s < 4; ++s)
        if (bc[s] < 0 || bc[s] > 2)
            return set_global_error(LBM2P_EINVAL, "unknown wall kind %d on side %d", bc[s], s);
    if ((bc[0] == LBM2P_BC_PERIODIC) != (bc[1] == LBM2P_BC_PERIODIC) ||
        (bc[2] == LBM2P_BC_PERIODIC) != (bc[3] == LBM2P_BC_PERIODIC))
        return set_global_error(LBM2P_EINVAL, "a periodic side must be paired with its opposite");
    for (int s = 0; s < 4; ++s)
        if (bc[s] == LBM2P_BC_DIRICHLET && (!P_b || !P_b[s] || (s < 2 ? nx : ny) < 3))
            return set_global_error(LBM2P_EINVAL, "Dirichlet side %d needs a wall trace and >= 3 nodes", s);
    for (int i = 0; i < 8; ++i)
        if (!n_in[i] || !n_out[i] || !aligned16(n_in[i]) || !aligned16(n_out[i]))
            return set_global_error(LBM2P_EINVAL, "population plane %d missing or not 16-byte aligned", i);
    if (!aligned16(R) || !aligned16(inv_tau) || !aligned16(dP) || (Fp && !aligned16(Fp)))
        return set_global_error(LBM2P_EINVAL, "R, inv_tau, dP and Fp must be 16-byte aligned");
    // the sweep reads its inputs while it writes its outputs: no output may be an input
    for (int i = 0; i < 8; ++i) {
        for (int j = 0; j < 8; ++j)
            if (n_out[i] == n_in[j])
                return set_global_error(LBM2P_EINVAL, "n_out[%d] is the same plane as n_in[%d]", i, j);
        if (n_out[i] == R || n_out[i] == inv_tau || n_out[i] == Fp || n_out[i] == dP)
            return set_global_error(LBM2P_EINVAL, "n_out[%d] aliases R, inv_tau, Fp or dP", i);
        for (int j = i + 1; j < 8; ++j)
            if (n_out[i] == n_out[j])
                return set_global_error(LBM2P_EINVAL, "n_out[%d] and n_out[%d] are the same plane", i, j);
    }
    for (int j = 0; j < 8; ++j)
        if (dP == n_in[j])
            return set_global_error(LBM2P_EINVAL, "dP is the same plane as n_in[%d]", j);
    if (dP == R || dP == inv_tau || dP == Fp)
        return set_global_error(LBM2P_EINVAL, "dP aliases R, inv_tau or Fp");

    double *scratch = nullptr;
    lbm2p_status st = scratch_on_current_device(&scratch);
    if (st != LBM2P_OK)
        return st;
    ResidualOut *out = reinterpret_cast<ResidualOut *>(scratch + kPartials);
    float *shift = reinterpret_cast<float *>(scratch + kPartials + kOutSlots);

    PressureArgs a{};
    for (int i = 0; i < 8; ++i) {
        a.fin[i] = n_in[i];
        a.fout[i] = n_out[i];
    }
    a.R = R;
    a.inv_tau = inv_tau;
    a.Fp = Fp;
    a.Pio = dP;
    a.partials = scratch;
    a.shift = shift;
    for (int s = 0; s < 4; ++s)
        a.Pb[s] = (P_b && bc[s] == LBM2P_BC_DIRICHLET) ? P_b[s] : nullptr;
    a.g.nx = nx;
    a.g.ny = ny;
    a.g.pitch = pitch;
    a.g.tiles_x = (nx + kBlock - 1) / kBlock;
    a.g.ntiles = a.g.tiles_x * ny;
    for (int s = 0; s < 4; ++s)
        a.g.bc[s] = bc[s];
    a.w.n = 0;

    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    // the two shifts start at zero on every call; the partials and the output are overwritten
    cudaError_t e = cudaMemsetAsync(shift, 0, 2 * sizeof(float), cs);
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "clearing the sweep scratch failed: %s", cudaGetErrorString(e));
    // one block per row tile, so every tile owns one slot of partials
    lbm2p_launch::pressure_sweep(a, true, true, (int)tiles, stream);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "pressure sweep launch failed: %s", cudaGetErrorString(e));
    lbm2p_launch::residual_finalize(scratch, (int)tiles, (long long)nx * ny, shift, out, stream);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "residual finalize launch failed: %s", cudaGetErrorString(e));
    double r = 0.0;
    e = cudaMemcpyAsync(&r, &out->r, sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess)
        return set_global_error(LBM2P_ECUDA, "reading the residual failed: %s", cudaGetErrorString(e));
    *residual = r;
    return LBM2P_OK;
}
