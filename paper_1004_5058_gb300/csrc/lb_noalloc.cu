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
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstdio>

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

// Device address of the scratch array on the current device.  Host code may
// not use the array's name as a device pointer; the address is looked up on
// every call (a host-side table lookup once the module is loaded), so nothing
// cached can outlive a device reset.
cudaError_t scratch_address(double** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

lb_status fail(lb_status st, const char* msg)
{
    char buf[320];
    snprintf(buf, sizeof buf, "lb_reductions_noalloc: %s", msg);
    set_handleless_error(buf);
    return st;
}

PFN_cuMemGetAddressRange_v3020 address_range_fn()
{
    static PFN_cuMemGetAddressRange_v3020 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 3020, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuMemGetAddressRange_v3020)p;
    }
    return fn;
}

}  // namespace

// A caller's buffer must be device (or managed) memory of the device `dev`
// whose allocation holds `bytes` bytes from `ptr` on; otherwise a kernel would
// read or write outside it.  Callers check before anything is launched.
bool lbhb::device_buffer_ok(const void* ptr, size_t bytes, int dev, const char* name, char* why, size_t why_len)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        snprintf(why, why_len, "%s: not a pointer the CUDA runtime knows", name);
        return false;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        snprintf(why, why_len, "%s: host memory; a device buffer of the current device is required", name);
        return false;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev) {
        snprintf(why, why_len, "%s: memory of device %d, the current device is %d", name, a.device, dev);
        return false;
    }
    auto range = address_range_fn();
    if (!range) {
        snprintf(why, why_len, "%s: cuMemGetAddressRange is not available", name);
        return false;
    }
    CUdeviceptr base = 0;
    size_t size = 0;
    if (range(&base, &size, (CUdeviceptr)(uintptr_t)ptr) != CUDA_SUCCESS) {
        snprintf(why, why_len, "%s: the extent of its allocation cannot be established", name);
        return false;
    }
    const uintptr_t p = (uintptr_t)ptr, end = (uintptr_t)base + size;
    if (p < (uintptr_t)base || p > end || bytes > end - p) {
        snprintf(why, why_len, "%s: %zu bytes needed from the pointer, its allocation holds %zu", name, bytes,
                 (size_t)(p <= end ? end - p : 0));
        return false;
    }
    return true;
}

namespace {

lb_status check_buffer(const void* ptr, size_t bytes, int dev, const char* name)
{
    char why[256];
    if (!device_buffer_ok(ptr, bytes, dev, name, why, sizeof why)) return fail(LB_ERR_INVALID, why);
    return LB_OK;
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
    // n_cells <= 16384 here, and g.plane < 2^62: the byte count needs no more than 2^61
    if (g.plane > (1LL << 61) / (18LL * elem * n_cells)) return fail(LB_ERR_INVALID, "buffer size overflows");
    const size_t pop_bytes = (size_t)n_cells * (size_t)g.cellstride * (size_t)elem;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "no usable current device");
    lb_status vs = check_buffer(populations, pop_bytes, dev, "populations");
    if (vs != LB_OK) return vs;
    vs = check_buffer(sums, (size_t)n_cells * 4 * sizeof(double), dev, "sums");
    if (vs != LB_OK) return vs;
    double* scratch = nullptr;
    e = scratch_address(&scratch);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, cudaGetErrorString(e));
    // the reduction kernels OR their non-finite/non-positive flag into this
    // word; this variant does not read it back (the sums of a cell with a
    // non-finite density are non-finite; a non-positive density is not flagged)
    unsigned* err = reinterpret_cast<unsigned*>(scratch + kScratchPartials);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (prec == LB_FP32)
        e = launch_state_sums<float>(static_cast<const float*>(populations), g, nullptr, scratch, sums, err, st);
    else
        e = launch_state_sums<double>(static_cast<const double*>(populations), g, nullptr, scratch, sums, err, st);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, cudaGetErrorString(e));
    return LB_OK;
}
