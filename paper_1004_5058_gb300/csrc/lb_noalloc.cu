// FP64 state reductions for callers that cannot allocate device memory.
//
// lb_reductions() works on a handle, and a handle owns device buffers that
// lb_create obtains with cudaMalloc, including the partial sums of the
// two-pass reduction.  Some callers cannot allocate: their device memory
// belongs to another allocator or to a fixed budget, or they cannot accept the
// implicit device-wide synchronisation that cudaMalloc/cudaFree may cause in a
// latency-critical loop.  lb_reductions_noalloc takes the populations and the
// output as the caller's own device buffers and runs the same two reduction
// kernels with their scratch (the per-block partial sums and the error word)
// in a fixed-size array compiled into the library.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "lbhb.h"
#include "lb_internal.h"

using namespace lbhb;

namespace {

// Capacity of the compiled-in scratch: partial sums (4 doubles per block and
// cell) plus one slot for the device error word.  512 KiB per GPU that loads
// the library, held until the process exits.
constexpr long long kScratchPartials = 65536;
constexpr long long kScratchDoubles = kScratchPartials + 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  Host code may
// not use the array's name as a device pointer, so the address is looked up
// once per device with cudaGetSymbolAddress, with that device current.
cudaError_t scratch_address(int dev, double** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

lb_status fail(lb_status st, const char* msg)
{
    char buf[320];
    snprintf(buf, sizeof buf, "lb_reductions_noalloc: %s", msg);
    set_handleless_error(buf);
    return st;
}

}  // namespace

extern "C" lb_status lb_reductions_noalloc(const void* populations, lb_precision prec, int nx, int ny, int pitch,
                                           int n_cells, double* sums, void* cuda_stream)
{
    if (!populations || !sums) return fail(LB_ERR_INVALID, "populations and sums must be device pointers");
    if (prec == LB_FP16_SHIFTED || prec == LB_FP16_SHIFTED_SR)
        return fail(LB_ERR_UNSUPPORTED, "FP16-shifted storage is not supported");
    if (prec != LB_FP32 && prec != LB_FP64) return fail(LB_ERR_INVALID, "unknown precision");
    if (nx < 1 || ny < 1 || n_cells < 1 || pitch < nx) return fail(LB_ERR_INVALID, "need nx, ny, n_cells >= 1, pitch >= nx");
    const int elem = prec == LB_FP64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(populations) % elem != 0 || reinterpret_cast<uintptr_t>(sums) % 8 != 0)
        return fail(LB_ERR_INVALID, "misaligned pointer");
    Geom g{};
    g.nx = nx;
    g.ny = ny;
    g.pitch = pitch;
    g.n_cells = n_cells;
    g.plane = (long long)ny * pitch;
    g.cellstride = 18 * g.plane;
    const long long need = (long long)n_cells * state_sums_blocks(g) * 4;
    if (need > kScratchPartials) {
        char buf[256];
        snprintf(buf, sizeof buf, "%d cells of %dx%d need %lld partial sums; the compiled-in scratch holds %lld",
                 n_cells, nx, ny, need, kScratchPartials);
        return fail(LB_ERR_INVALID, buf);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(LB_ERR_CUDA, "no usable current device");
    double* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, cudaGetErrorString(e));
    unsigned* err = reinterpret_cast<unsigned*>(scratch + kScratchPartials);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the error word is the only scratch read before it is written
    e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        if (prec == LB_FP32)
            e = launch_state_sums<float>(static_cast<const float*>(populations), g, nullptr, scratch, sums, err, st);
        else
            e = launch_state_sums<double>(static_cast<const double*>(populations), g, nullptr, scratch, sums, err, st);
    }
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, cudaGetErrorString(e));
    return LB_OK;
}
