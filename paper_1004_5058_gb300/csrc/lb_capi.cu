// C ABI of the library (declared in include/lbhb.h): handle life cycle,
// argument validation, device memory, the step loop (with CUDA graphs for
// chunks of steps), observables and error reporting.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "lbhb.h"
#include "lb_internal.h"

using namespace lbhb;

// NVTX range around a C ABI call, for timeline tools (a no-op without one)
struct Trace {
    explicit Trace(const char* name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
};

struct lb_handle {
    int n_cells = 0, nx = 0, ny = 0, bc = 0;
    lb_precision prec = LB_FP32;
    int elem = 4;
    std::vector<lb_cell_params> cells;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Geom g{};                          // the rows a step updates: ny = own rows (the whole cell, or a slab)
    Geom gbuf{};                       // the whole population buffer (a slab adds two ghost rows each side)
    RowMap rm{};
    long long view_off = 0;            // elements from a buffer's start to row 0 of g
    bool slab = false;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* aux = nullptr;               // generic family: rho/psi field
    double* prof_part = nullptr;       // [cell][nbx][ny] partials of one sampled step
    double* wall_part = nullptr;       // [cell][nbx][2]
    int nbx_alloc = 0;
    double* acc_prof = nullptr;        // [cell][ny] time sums of the line profile
    double* acc_wall = nullptr;        // [cell][2] time sums of Pi_top, Pi_bot
    unsigned* d_err = nullptr;
    unsigned* h_err = nullptr;         // pinned mirror of d_err at the end of the last batch
    cudaEvent_t batch_done = nullptr;
    bool batch_pending = false;
    CellDev* d_cells = nullptr;
    double* red_part = nullptr;
    double* red_out = nullptr;
    double* staging = nullptr;         // [cell][4][ny][nx] float64
    cudaStream_t copy_stream = nullptr;  // lb_stage_fields' copies (created on first use)
    cudaEvent_t staged = nullptr;        // the last staged copy is complete
    cudaEvent_t staging_read = nullptr;  // the last equilibrium launch has read the staging buffer
    bool staged_pending = false;         // fields staged and not yet consumed
    long long t = 0, start = 0, every = 0, n_samples = 0;
    bool initialised = false;
    bool faulted = false;
    bool use_graphs = true;
    lb_kernel kernel = LB_KERNEL_GENERIC;
    int tile_x = 0, tile_y = 0;
    TiledPlan* plan = nullptr;
    long long launches = 0;
    int inject = 0;  // lb_test_inject: 1 = stalled row copy, 2 = failed launch (next lb_step)
    std::string last_error;
    // CUDA graphs of step chunks, keyed by (source buffer, steps, sampled last step)
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
};

static const char* g_null_msg = "lb: handle is NULL";
static thread_local char g_create_msg[512] = "";

void lbhb::set_handleless_error(const char* msg) { snprintf(g_create_msg, sizeof g_create_msg, "%s", msg); }

static lb_status fail(lb_handle* h, lb_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->last_error = buf;
    else snprintf(g_create_msg, sizeof g_create_msg, "%s", buf);
    return st;
}

#define CK(h, call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail((h), LB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void free_graphs(lb_handle* h)
{
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

static void release(lb_handle* h)
{
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_graphs(h);
    if (h->plan) tiled_destroy(h->plan);
    cudaFree(h->f[0]);
    cudaFree(h->f[1]);
    cudaFree(h->aux);
    cudaFree(h->prof_part);
    cudaFree(h->wall_part);
    cudaFree(h->acc_prof);
    cudaFree(h->acc_wall);
    cudaFree(h->d_err);
    cudaFree(h->d_cells);
    cudaFree(h->red_part);
    cudaFree(h->red_out);
    cudaFree(h->staging);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->batch_done) cudaEventDestroy(h->batch_done);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    if (h->staged) cudaEventDestroy(h->staged);
    if (h->staging_read) cudaEventDestroy(h->staging_read);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    cudaSetDevice(prev);
    delete h;
}

// true if the cell sets a multiple-relaxation-time rate
static bool has_mrt(const lb_cell_params& c) { return c.s_e != 0.0 || c.s_eps != 0.0 || c.s_q != 0.0 || c.s_nu != 0.0; }

template <class C>
static void fill(ParamSet<C>& d, const lb_cell_params& c)
{
    const double tau_b = c.tau_b == 0.0 ? c.tau : c.tau_b;
    d.tau = C(c.tau);
    d.omega = C(1.0 / c.tau);
    d.tau_b = C(tau_b);
    d.omega_b = C(1.0 / tau_b);
    d.mix[0] = C(c.tau / tau_b);
    d.mix[1] = C(tau_b / c.tau);
    d.rho0 = C(c.rho0);
    d.inv_rho0 = C(1.0 / c.rho0);
    d.gab_over_rho0 = C(c.g_ab / c.rho0);
    d.g1[0] = C(c.g_aa1);
    d.g1[1] = C(c.g_bb1);
    d.g2[0] = C(c.g_aa2);
    d.g2[1] = C(c.g_bb2);
    d.u_wall = C(c.u_wall);
    d.f0 = C(c.f0);
    d.two_over_ny = C(2.0 / c.ny);
    d.rho_bar[0] = C(c.rho_bar_a);
    d.rho_bar[1] = C(c.rho_bar_b);
    // multiple relaxation times: (w - s_k)/D per species, s_k = w where unset
    d.mrt = has_mrt(c) ? 1 : 0;
    for (int s = 0; s < 2; ++s) {
        const double w = 1.0 / (s ? tau_b : c.tau);
        const double r[4] = {c.s_e, c.s_eps, c.s_q, c.s_nu}, norm[4] = {12.0, 12.0, 12.0, 4.0};
        for (int k = 0; k < 4; ++k) d.mrt_h[s][k] = C(d.mrt ? (w - (r[k] != 0.0 ? r[k] : w)) / norm[k] : 0.0);
    }
}

// The batch's collision for the tiled kernels: MRT if any cell sets a rate,
// else BGK with one relaxation time unless some cell gives species B its own
static int collision_kind(const std::vector<lb_cell_params>& cells)
{
    int kind = TILED_BGK_ONE_TIME;
    for (const lb_cell_params& c : cells) {
        if (has_mrt(c)) return TILED_MRT;
        if (c.tau_b != 0.0 && c.tau_b != c.tau) kind = TILED_BGK;
    }
    return kind;
}

static CellDev to_dev(const lb_cell_params& c)
{
    CellDev d{};
    fill(d.d, c);
    fill(d.f, c);
    return d;
}

// Dispatch on the storage type.
template <class F>
static cudaError_t with_type(const lb_handle* h, F&& fn)
{
    switch (h->prec) {
    case LB_FP32: return fn((float*)nullptr);
    case LB_FP64: return fn((double*)nullptr);
    case LB_FP16_SHIFTED_SR: return fn((half_sr*)nullptr);
    default: return fn((__half*)nullptr);
    }
}

// Buffer b at row 0 of the updated rows (the whole buffer for a whole cell).
static void* fview(const lb_handle* h, int b) { return (char*)h->f[b] + h->view_off * h->elem; }

static lb_status check_device_error(lb_handle* h)
{
    unsigned e = 0;
    CK(h, cudaMemcpy(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost));
    if (e & ERR_NONFINITE) {
        h->faulted = true;
        return fail(h, LB_ERR_NONFINITE, "lb: non-finite or non-positive density detected on the device");
    }
    if (e & ERR_TIMEOUT) {
        h->faulted = true;
        return fail(h, LB_ERR_TIMEOUT, "lb: a bounded device wait ran out (pipeline stalled)");
    }
    return LB_OK;
}

static lb_status sync_and_check(lb_handle* h)
{
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    h->batch_pending = false;
    return check_device_error(h);
}

static lb_status reset_counters(lb_handle* h)
{
    h->t = 0;
    h->n_samples = 0;
    h->faulted = false;
    h->initialised = true;
    CK(h, cudaMemsetAsync(h->acc_prof, 0, sizeof(double) * h->n_cells * h->ny, h->stream));
    CK(h, cudaMemsetAsync(h->acc_wall, 0, sizeof(double) * h->n_cells * 2, h->stream));
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream));
    h->h_err[0] = 0;
    return LB_OK;
}

static lb_status select_kernel(lb_handle* h, lb_kernel k, int tx, int ty)
{
    if (k == LB_KERNEL_AUTO) {
        // the widest tile that divides nx, else the widest that fits (a narrower
        // last strip), else the generic kernel
        const int txs[] = {128, 64, 32};
        for (int pass = 0; pass < 2; ++pass)
            for (int c : txs)
                if ((pass == 1 || h->nx % c == 0) && tiled_supported(h->gbuf, h->elem, c, 0) &&
                    select_kernel(h, LB_KERNEL_TILED, c, 0) == LB_OK)
                    return LB_OK;
        return select_kernel(h, LB_KERNEL_GENERIC, 0, 0);
    }
    if (k == LB_KERNEL_GENERIC && h->slab)
        return fail(h, LB_ERR_UNSUPPORTED, "lb_set_kernel: a slab runs the tiled kernel only");
    free_graphs(h);
    if (k == LB_KERNEL_GENERIC) {
        if (h->plan) {
            tiled_destroy(h->plan);
            h->plan = nullptr;
        }
        h->kernel = LB_KERNEL_GENERIC;
        h->tile_x = 32;
        h->tile_y = 8;
        return LB_OK;
    }
    if (k != LB_KERNEL_TILED) return fail(h, LB_ERR_INVALID, "lb_set_kernel: unknown kernel %d", (int)k);
    if (tx == 0) {
        tx = 32;
        for (int c : {128, 64})
            if (h->nx % c == 0) {
                tx = c;
                break;
            }
    }
    if (!tiled_supported(h->gbuf, h->elem, tx, ty))
        return fail(h, LB_ERR_UNSUPPORTED, "lb_set_kernel: tiled kernel does not support nx=%d ny=%d tile %dx%d",
                    h->nx, h->ny, tx, ty);
    if (tiled_partials_nbx(h->g, tx) > h->nbx_alloc)
        return fail(h, LB_ERR_UNSUPPORTED, "lb_set_kernel: tile %d too narrow for the partial buffers", tx);
    const char* msg = nullptr;
    TiledPlan* p = tiled_create(h->gbuf, h->rm, (int)h->prec, h->elem, h->bc, h->f[0], h->f[1], tx, ty, &msg);
    if (!p) return fail(h, LB_ERR_UNSUPPORTED, "lb_set_kernel: %s", msg ? msg : "tiled plan failed");
    tiled_set_collision(p, collision_kind(h->cells));
    if (h->plan) tiled_destroy(h->plan);
    h->plan = p;
    h->kernel = LB_KERNEL_TILED;
    tiled_tiles(p, &h->tile_x, &h->tile_y);
    return LB_OK;
}

// ------------------------------------------------------------ checkpoints --
// File layout (version 3, this machine's byte order):
//   header  128 bytes: magic "LBHBCKPT", u32 version, u32 header bytes, i32
//           n_cells, nx, ny, bc, precision, element bytes, i64 t, start,
//           every, n_samples, u64 payload bytes, u64 FNV-1a 64 of the payload
//   payload 19 float64 per cell (lb_cell_params in declaration order; version
//           2 files hold the first 15, without the MRT rates, and load them as
//           0; version 1 files the first 14, also without tau_b), the
//           time sums of the line profile [cell][ny] and of the wall momenta
//           [cell][2] (float64), the populations [cell][s][i][y][x] in the
//           storage precision without row padding
namespace {

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t n_cells, nx, ny, bc, prec, elem;
    int64_t t, start, every, n_samples;
    uint64_t payload_bytes, checksum;
    unsigned char pad[128 - 8 - 8 - 24 - 32 - 16];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header layout");

const char kMagic[8] = {'L', 'B', 'H', 'B', 'C', 'K', 'P', 'T'};

// FNV-1a, 64-bit (Fowler, Noll, Vo)
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n)
    {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t k = 0; k < n; ++k) h = (h ^ b[k]) * 1099511628211ull;
    }
};

constexpr int kCellDoubles = 19;  // per cell in version 3 (15 in version 2, 14 in version 1)

void cell_to_doubles(const lb_cell_params& c, double v[kCellDoubles])
{
    const double a[kCellDoubles] = {(double)c.nx, (double)c.ny, c.tau, c.rho0, c.g_aa1, c.g_aa2, c.g_bb1,
                                    c.g_bb2, c.g_ab, c.u_wall, c.f0, c.rho_bar_a, c.rho_bar_b, (double)c.bc,
                                    c.tau_b, c.s_e, c.s_eps, c.s_q, c.s_nu};
    for (int k = 0; k < kCellDoubles; ++k) v[k] = a[k];
}

// false if the integer fields are not small whole numbers; fields a file's
// version does not hold arrive as 0 (tau_b, the MRT rates)
bool cell_from_doubles(const double v[kCellDoubles], lb_cell_params* out)
{
    for (int k : {0, 1, 13})
        if (!(v[k] >= 0.0 && v[k] <= 2147483647.0) || v[k] != std::floor(v[k])) return false;
    lb_cell_params& c = *out;
    c.nx = (int)v[0];
    c.ny = (int)v[1];
    c.tau = v[2];
    c.rho0 = v[3];
    c.g_aa1 = v[4];
    c.g_aa2 = v[5];
    c.g_bb1 = v[6];
    c.g_bb2 = v[7];
    c.g_ab = v[8];
    c.u_wall = v[9];
    c.f0 = v[10];
    c.rho_bar_a = v[11];
    c.rho_bar_b = v[12];
    c.bc = (lb_bc)(int)v[13];
    c.tau_b = v[14];
    c.s_e = v[15];
    c.s_eps = v[16];
    c.s_q = v[17];
    c.s_nu = v[18];
    return true;
}

struct File {
    FILE* f = nullptr;
    ~File()
    {
        if (f) fclose(f);
    }
};

}  // namespace

// Cells a handle can run: one shape and boundary kind, tau > 1/2, rho0 > 0,
// finite couplings.  On failure writes the reason to why.
static bool cells_valid(const lb_cell_params* cells, int n_cells, char* why, size_t n)
{
    const lb_cell_params& c0 = cells[0];
    for (int c = 0; c < n_cells; ++c) {
        const lb_cell_params& p = cells[c];
        if (p.nx != c0.nx || p.ny != c0.ny || p.bc != c0.bc) {
            snprintf(why, n, "cell %d differs in nx/ny/bc from cell 0", c);
            return false;
        }
        if (p.nx < 5 || p.ny < 5 || (long long)p.nx * p.ny > (1LL << 31)) {
            snprintf(why, n, "lattice %dx%d out of range (5 .. 2^31 sites)", p.nx, p.ny);
            return false;
        }
        if (!(p.tau > 0.5) || !std::isfinite(p.tau)) {
            snprintf(why, n, "cell %d tau=%g must exceed 1/2", c, p.tau);
            return false;
        }
        if (p.tau_b != 0.0 && (!(p.tau_b > 0.5) || !std::isfinite(p.tau_b))) {
            snprintf(why, n, "cell %d tau_b=%g must exceed 1/2 (or be 0: tau)", c, p.tau_b);
            return false;
        }
        for (double r : {p.s_e, p.s_eps, p.s_q, p.s_nu})
            if (r != 0.0 && !(r > 0.0 && r < 2.0)) {
                snprintf(why, n, "cell %d: a multiple-relaxation-time rate %g is outside (0, 2) (0: 1/tau)", c, r);
                return false;
            }
        if (!(p.rho0 > 0.0) || !std::isfinite(p.rho0)) {
            snprintf(why, n, "cell %d rho0=%g must be positive", c, p.rho0);
            return false;
        }
        if (p.bc != LB_BC_PERIODIC && p.bc != LB_BC_COUETTE) {
            snprintf(why, n, "unknown boundary %d", p.bc);
            return false;
        }
        const double v[] = {p.g_aa1, p.g_aa2, p.g_bb1, p.g_bb2, p.g_ab, p.u_wall, p.f0, p.rho_bar_a, p.rho_bar_b};
        for (double x : v)
            if (!std::isfinite(x)) {
                snprintf(why, n, "cell %d has a non-finite parameter", c);
                return false;
            }
    }
    return true;
}

// A handle over the whole cells (rows < 0), or over rows [y0, y0 + rows) of
// each cell with two ghost rows on each side (a slab).
static lb_status create_handle(const lb_cell_params* cells, int n_cells, lb_precision prec, void* cuda_stream,
                               int y0, int rows, lb_handle** out)
{
    if (!out) return fail(nullptr, LB_ERR_INVALID, "lb_create: out is NULL");
    *out = nullptr;
    if (!cells || n_cells < 1) return fail(nullptr, LB_ERR_INVALID, "lb_create: need n_cells >= 1 cells");
    if (prec != LB_FP32 && prec != LB_FP16_SHIFTED && prec != LB_FP64 && prec != LB_FP16_SHIFTED_SR)
        return fail(nullptr, LB_ERR_INVALID, "lb_create: unknown precision %d", (int)prec);
    char why[256];
    if (!cells_valid(cells, n_cells, why, sizeof why)) return fail(nullptr, LB_ERR_INVALID, "lb_create: %s", why);
    const lb_cell_params& c0 = cells[0];
    const bool slab = rows >= 0;
    if (slab) {
        if (rows < 2 || y0 < 0 || (long long)y0 + rows > c0.ny)
            return fail(nullptr, LB_ERR_INVALID, "lb_create_slab: rows [%d, %d) do not fit a cell of %d rows (and a "
                        "slab needs at least 2)", y0, y0 + rows, c0.ny);
        if (c0.bc == LB_BC_PERIODIC && rows + 4 > c0.ny)
            return fail(nullptr, LB_ERR_INVALID, "lb_create_slab: a periodic cell of %d rows cannot hold a slab of "
                        "%d rows and its four ghost rows", c0.ny, rows);
    }
    lb_handle* h = new (std::nothrow) lb_handle();
    if (!h) return fail(nullptr, LB_ERR_NOMEM, "lb_create: out of host memory");
    h->n_cells = n_cells;
    h->nx = c0.nx;
    h->ny = slab ? rows : c0.ny;  // the rows a step updates
    h->bc = c0.bc;
    h->slab = slab;
    h->prec = prec;
    h->elem = prec == LB_FP64 ? 8 : (prec == LB_FP32 ? 4 : 2);
    h->cells.assign(cells, cells + n_cells);
    cudaError_t e = cudaGetDevice(&h->device);
    auto bail = [&](lb_status st, const char* what, cudaError_t ce) {
        fail(nullptr, st, "lb_create: %s: %s", what, cudaGetErrorString(ce));
        release(h);
        return st;
    };
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, "cudaGetDevice", e);
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(LB_ERR_CUDA, "cudaStreamCreate", e);
        h->own_stream = true;
    }
    const int align = 128 / h->elem;  // rows start on 128-byte boundaries
    h->gbuf.nx = h->nx;
    h->gbuf.ny = slab ? rows + 4 : h->ny;
    h->gbuf.pitch = (h->nx + align - 1) / align * align;
    h->gbuf.n_cells = n_cells;
    h->gbuf.plane = (long long)h->gbuf.ny * h->gbuf.pitch;
    h->gbuf.cellstride = 18 * h->gbuf.plane;
    h->g = h->gbuf;  // the updated rows as a view of the buffer: same strides, fewer rows
    h->g.ny = h->ny;
    h->view_off = slab ? 2LL * h->gbuf.pitch : 0;
    h->rm.ylo = slab ? 2 : 0;
    h->rm.nown = h->ny;
    h->rm.y0g = slab ? y0 : 0;
    h->rm.nyg = c0.ny;
    h->rm.slab = slab ? 1 : 0;
    const size_t fbytes = (size_t)n_cells * h->gbuf.cellstride * h->elem;
    const size_t n = (size_t)h->nx * h->ny;
    const size_t cbytes = prec == LB_FP64 ? 8 : 4;
    h->nbx_alloc = std::max(generic_partials_nbx(h->g), tiled_partials_nbx(h->g, 32));
    struct A { void** p; size_t b; } allocs[] = {
        {&h->f[0], fbytes},
        {&h->f[1], fbytes},
        {&h->aux, (size_t)n_cells * 4 * n * cbytes},
        {(void**)&h->prof_part, sizeof(double) * n_cells * h->nbx_alloc * h->ny},
        {(void**)&h->wall_part, sizeof(double) * n_cells * h->nbx_alloc * 2},
        {(void**)&h->acc_prof, sizeof(double) * n_cells * h->ny},
        {(void**)&h->acc_wall, sizeof(double) * n_cells * 2},
        {(void**)&h->d_err, sizeof(unsigned)},
        {(void**)&h->d_cells, sizeof(CellDev) * n_cells},
        {(void**)&h->red_part, sizeof(double) * n_cells * state_sums_blocks(h->g) * 4},
        {(void**)&h->red_out, sizeof(double) * n_cells * 4},
    };
    for (auto& a : allocs) {
        e = cudaMalloc(a.p, a.b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA, "cudaMalloc", e);
        }
    }
    e = cudaHostAlloc((void**)&h->h_err, sizeof(unsigned), cudaHostAllocDefault);
    if (e != cudaSuccess) return bail(LB_ERR_NOMEM, "cudaHostAlloc", e);
    e = cudaEventCreateWithFlags(&h->batch_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, "cudaEventCreate", e);
    std::vector<CellDev> dc(n_cells);
    for (int c = 0; c < n_cells; ++c) dc[c] = to_dev(cells[c]);
    e = cudaMemcpyAsync(h->d_cells, dc.data(), sizeof(CellDev) * n_cells, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, fbytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[1], 0, fbytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->prof_part, 0, sizeof(double) * n_cells * h->nbx_alloc * h->ny, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->wall_part, 0, sizeof(double) * n_cells * h->nbx_alloc * 2, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, "initial copies", e);
    if (reset_counters(h) != LB_OK) {
        fail(nullptr, LB_ERR_CUDA, "lb_create: %s", h->last_error.c_str());
        release(h);
        return LB_ERR_CUDA;
    }
    h->initialised = false;
    const lb_status ks = select_kernel(h, LB_KERNEL_AUTO, 0, 0);
    if (ks != LB_OK) {
        // a slab runs the tiled kernel only: a shape it does not take is unsupported
        const lb_status st = ks == LB_ERR_UNSUPPORTED ? LB_ERR_UNSUPPORTED : LB_ERR_CUDA;
        fail(nullptr, st, "%s: %s", slab ? "lb_create_slab" : "lb_create", h->last_error.c_str());
        release(h);
        return st;
    }
    *out = h;
    return LB_OK;
}

extern "C" {

lb_status lb_create(const lb_cell_params* cells, int n_cells, lb_precision prec, void* cuda_stream,
                    lb_handle** out)
{
    return create_handle(cells, n_cells, prec, cuda_stream, 0, -1, out);
}

lb_status lb_create_slab(const lb_cell_params* cells, int n_cells, lb_precision prec, int y0, int rows,
                         void* cuda_stream, lb_handle** out)
{
    if (rows < 0) return fail(nullptr, LB_ERR_INVALID, "lb_create_slab: rows < 0");
    return create_handle(cells, n_cells, prec, cuda_stream, y0, rows, out);
}

lb_status lb_init_fields(lb_handle* h, const double* rho_a, const double* rho_b, const double* ux,
                         const double* uy)
{
    Trace trace("lb_init_fields");
    if (!h) return LB_ERR_INVALID;
    if (!rho_a || !rho_b) return fail(h, LB_ERR_INVALID, "lb_init_fields: rho_a and rho_b are required");
    CK(h, cudaSetDevice(h->device));
    const size_t n = (size_t)h->nx * h->ny;
    if (!h->staging) CK(h, cudaMalloc(&h->staging, sizeof(double) * 4 * n * h->n_cells));
    if (h->copy_stream) {  // a staged copy in flight writes the same buffer: let it land, then drop it
        CK(h, cudaStreamSynchronize(h->copy_stream));
        h->staged_pending = false;
    }
    const double* src[4] = {rho_a, rho_b, ux, uy};
    for (int a = 0; a < 4; ++a) {
        double* dst = h->staging + a * n;
        if (src[a])
            CK(h, cudaMemcpy2DAsync(dst, 4 * n * sizeof(double), src[a], n * sizeof(double), n * sizeof(double),
                                    h->n_cells, cudaMemcpyHostToDevice, h->stream));
        else
            CK(h, cudaMemset2DAsync(dst, 4 * n * sizeof(double), 0, n * sizeof(double), h->n_cells, h->stream));
    }
    CK(h, with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        return launch_equilibrium<T>(h->staging, (T*)fview(h, 0), h->g, h->d_cells, h->stream);
    }));
    h->launches += 1;
    h->cur = 0;
    lb_status st = reset_counters(h);
    if (st != LB_OK) return st;
    CK(h, cudaStreamSynchronize(h->stream));
    h->batch_pending = false;
    return LB_OK;
}

lb_status lb_stage_fields(lb_handle* h, const double* rho_a, const double* rho_b, const double* ux,
                          const double* uy)
{
    Trace trace("lb_stage_fields");
    if (!h) return LB_ERR_INVALID;
    if (!rho_a || !rho_b) return fail(h, LB_ERR_INVALID, "lb_stage_fields: rho_a and rho_b are required");
    CK(h, cudaSetDevice(h->device));
    const size_t n = (size_t)h->nx * h->ny;
    if (!h->staging) {
        cudaError_t e = cudaMalloc(&h->staging, sizeof(double) * 4 * n * h->n_cells);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->staging = nullptr;
            return fail(h, LB_ERR_NOMEM, "lb_stage_fields: staging buffer: %s", cudaGetErrorString(e));
        }
    }
    if (!h->copy_stream) {  // all three or none, so a failed set-up leaves nothing half made
        cudaStream_t cs = nullptr;
        cudaEvent_t done = nullptr, read = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&read, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(read, h->stream);  // nothing has read the buffer yet
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (read) cudaEventDestroy(read);
            if (done) cudaEventDestroy(done);
            if (cs) cudaStreamDestroy(cs);
            return fail(h, LB_ERR_CUDA, "lb_stage_fields: copy stream: %s", cudaGetErrorString(e));
        }
        h->copy_stream = cs;
        h->staged = done;
        h->staging_read = read;
    }
    // the buffer is free once the last equilibrium launch that reads it has run
    CK(h, cudaStreamWaitEvent(h->copy_stream, h->staging_read, 0));
    const double* src[4] = {rho_a, rho_b, ux, uy};
    for (int a = 0; a < 4; ++a) {
        double* dst = h->staging + a * n;
        if (src[a])
            CK(h, cudaMemcpy2DAsync(dst, 4 * n * sizeof(double), src[a], n * sizeof(double), n * sizeof(double),
                                    h->n_cells, cudaMemcpyHostToDevice, h->copy_stream));
        else
            CK(h, cudaMemset2DAsync(dst, 4 * n * sizeof(double), 0, n * sizeof(double), h->n_cells,
                                    h->copy_stream));
    }
    CK(h, cudaEventRecord(h->staged, h->copy_stream));
    h->staged_pending = true;
    return LB_OK;
}

lb_status lb_init_fields_staged(lb_handle* h)
{
    Trace trace("lb_init_fields_staged");
    if (!h) return LB_ERR_INVALID;
    if (!h->staged_pending) return fail(h, LB_ERR_STATE, "lb_init_fields_staged: no fields staged (lb_stage_fields)");
    CK(h, cudaSetDevice(h->device));
    // the host arrays are free once this returns; an earlier batch's error mirror
    // lands before the counters below are reset
    CK(h, cudaEventSynchronize(h->staged));
    if (h->batch_pending) {
        CK(h, cudaEventSynchronize(h->batch_done));
        h->batch_pending = false;
    }
    h->staged_pending = false;
    CK(h, cudaStreamWaitEvent(h->stream, h->staged, 0));
    CK(h, with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        return launch_equilibrium<T>(h->staging, (T*)fview(h, 0), h->g, h->d_cells, h->stream);
    }));
    CK(h, cudaEventRecord(h->staging_read, h->stream));
    h->launches += 1;
    h->cur = 0;
    return reset_counters(h);
}

lb_status lb_set_populations(lb_handle* h, const double* f)
{
    Trace trace("lb_set_populations");
    if (!h) return LB_ERR_INVALID;
    if (!f) return fail(h, LB_ERR_INVALID, "lb_set_populations: f is NULL");
    CK(h, cudaSetDevice(h->device));
    const size_t bytes = sizeof(double) * 18 * (size_t)h->nx * h->ny * h->n_cells;
    double* tmp = nullptr;
    CK(h, cudaMalloc(&tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = with_type(h, [&](auto* tp) {
            using T = std::remove_pointer_t<decltype(tp)>;
            return launch_import<T>(tmp, (T*)fview(h, 0), h->g, h->d_cells, h->stream);
        });
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(h, LB_ERR_CUDA, "lb_set_populations: %s", cudaGetErrorString(e));
    h->launches += 1;
    h->cur = 0;
    lb_status st = reset_counters(h);
    if (st != LB_OK) return st;
    CK(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

lb_status lb_get_populations(lb_handle* h, double* f)
{
    Trace trace("lb_get_populations");
    if (!h) return LB_ERR_INVALID;
    if (!f) return fail(h, LB_ERR_INVALID, "lb_get_populations: f is NULL");
    if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_get_populations: no state loaded");
    CK(h, cudaSetDevice(h->device));
    const size_t bytes = sizeof(double) * 18 * (size_t)h->nx * h->ny * h->n_cells;
    double* tmp = nullptr;
    CK(h, cudaMalloc(&tmp, bytes));
    cudaError_t e = with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        return launch_export<T>((const T*)fview(h, h->cur), tmp, h->g, h->d_cells, h->stream);
    });
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(h, LB_ERR_CUDA, "lb_get_populations: %s", cudaGetErrorString(e));
    h->launches += 1;
    return LB_OK;
}

static cudaError_t enqueue_one_step(lb_handle* h, int src, bool sample, int* nl)
{
    cudaError_t e = with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        if (h->kernel == LB_KERNEL_TILED)
            return launch_tiled_step<T>(h->plan, src, h->d_cells, sample, h->prof_part, h->wall_part, h->d_err,
                                        h->stream, nl);
        return launch_generic_step<T>((const T*)h->f[src], (T*)h->f[1 - src], h->g, h->bc, h->d_cells, h->aux,
                                      sample, h->prof_part, h->wall_part, h->d_err, h->stream, nl);
    });
    if (e != cudaSuccess || !sample) return e;
    const int nbx = h->kernel == LB_KERNEL_TILED ? tiled_partials_nbx(h->g, h->tile_x) : generic_partials_nbx(h->g);
    *nl += 1;
    return launch_accumulate(h->prof_part, h->wall_part, nbx, h->ny, h->bc, h->n_cells, h->acc_prof, h->acc_wall,
                             h->stream);
}

// A chunk of `steps` steps starting from buffer `src`; only the last one may be sampled.
static cudaError_t run_chunk(lb_handle* h, int src, int steps, bool sample_last, int* nl)
{
    const int min_graph = 4;
    if (steps < min_graph) {
        for (int k = 0; k < steps; ++k) {
            cudaError_t e = enqueue_one_step(h, src, sample_last && k == steps - 1, nl);
            if (e != cudaSuccess) return e;
            src ^= 1;
        }
        return cudaSuccess;
    }
    auto key = std::make_tuple(src, steps, sample_last ? 1 : 0);
    auto it = h->graphs.find(key);
    int per = 0;
    if (it == h->graphs.end()) {
        if (h->graphs.size() > 64) free_graphs(h);
        cudaGraph_t graph = nullptr;
        cudaError_t e = h->use_graphs ? cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)
                                      : cudaErrorStreamCaptureUnsupported;
        if (e != cudaSuccess) {
            // streams that cannot be captured (the legacy default stream): plain launches
            cudaGetLastError();
            h->use_graphs = false;
            for (int k = 0; k < steps; ++k) {
                e = enqueue_one_step(h, src, sample_last && k == steps - 1, nl);
                if (e != cudaSuccess) return e;
                src ^= 1;
            }
            return cudaSuccess;
        }
        int s = src;
        for (int k = 0; k < steps && e == cudaSuccess; ++k) {
            e = enqueue_one_step(h, s, sample_last && k == steps - 1, &per);
            s ^= 1;
        }
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return e;
        }
        if (e2 != cudaSuccess) return e2;
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return e;
        it = h->graphs.emplace(key, exec).first;
    }
    // count the launches the graph holds
    int kernels_per_step = h->kernel == LB_KERNEL_TILED ? 1 : 2;
    *nl += steps * kernels_per_step + (sample_last ? 1 : 0);
    return cudaGraphLaunch(it->second, h->stream);
}

lb_status lb_step(lb_handle* h, long long n_steps)
{
    Trace trace("lb_step");
    if (!h) return LB_ERR_INVALID;
    if (n_steps < 0) return fail(h, LB_ERR_INVALID, "lb_step: n_steps < 0");
    if (h->slab && n_steps > 1)
        return fail(h, LB_ERR_INVALID, "lb_step: a slab takes one step per call (its ghost rows and the populations "
                    "that left it are traded between steps)");
    if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_step: no state loaded (call lb_init_fields)");
    if (h->faulted) return fail(h, LB_ERR_STATE, "lb_step: an earlier device error left the state invalid");
    CK(h, cudaSetDevice(h->device));
    if (h->batch_pending && cudaEventQuery(h->batch_done) == cudaSuccess) {
        h->batch_pending = false;
        if (h->h_err[0]) {
            h->faulted = true;
            return fail(h, (h->h_err[0] & ERR_TIMEOUT) ? LB_ERR_TIMEOUT : LB_ERR_NONFINITE,
                        "lb_step: the previous batch reported a device error (%u)", h->h_err[0]);
        }
    }
    if (n_steps == 0) return LB_OK;
    if (h->inject == 2) {
        h->inject = 0;
        return fail(h, LB_ERR_CUDA, "lb_step: launch failed: injected failure (lb_test_inject)");
    }
    int nl = 0;
    long long done = 0;
    while (done < n_steps) {
        // steps up to and including the next sampled step (or the end)
        long long left = n_steps - done;
        long long to_sample = -1;
        if (h->every > 0) {
            long long t = h->t;
            long long next = t <= h->start ? h->start : h->start + ((t - h->start + h->every - 1) / h->every) * h->every;
            to_sample = next - t;  // steps before the sampled one
        }
        long long chunk;
        bool sample_last = false;
        if (to_sample >= 0 && to_sample < left) {
            chunk = to_sample + 1;
            sample_last = true;
        } else {
            chunk = left;
        }
        // split long unsampled runs into graph-sized pieces
        while (chunk > 0) {
            const long long piece_max = 64;
            // an injected stall applies to one plain launch, never to a captured graph
            const bool stall = h->inject == 1 && h->plan != nullptr;
            const long long piece = stall ? 1 : (chunk > piece_max ? piece_max : chunk);
            const bool s_last = sample_last && piece == chunk;
            cudaError_t e;
            if (stall) {
                h->inject = 0;
                tiled_inject_skip(h->plan, 5);
                e = enqueue_one_step(h, h->cur, s_last, &nl);
            } else {
                e = run_chunk(h, h->cur, (int)piece, s_last, &nl);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(h, LB_ERR_CUDA, "lb_step: launch failed: %s", cudaGetErrorString(e));
            }
            if (piece & 1) h->cur ^= 1;
            h->t += piece;
            done += piece;
            chunk -= piece;
            if (s_last) h->n_samples += 1;
        }
    }
    h->launches += nl;
    CK(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaEventRecord(h->batch_done, h->stream));
    h->batch_pending = true;
    return LB_OK;
}

lb_status lb_set_sampling(lb_handle* h, long long start_step, long long every)
{
    if (!h) return LB_ERR_INVALID;
    if (every < 0 || start_step < 0) return fail(h, LB_ERR_INVALID, "lb_set_sampling: negative argument");
    CK(h, cudaSetDevice(h->device));
    h->start = start_step;
    h->every = every;
    h->n_samples = 0;
    CK(h, cudaMemsetAsync(h->acc_prof, 0, sizeof(double) * h->n_cells * h->ny, h->stream));
    CK(h, cudaMemsetAsync(h->acc_wall, 0, sizeof(double) * h->n_cells * 2, h->stream));
    return LB_OK;
}

static lb_status read_acc(lb_handle* h, std::vector<double>& prof, std::vector<double>& wall)
{
    lb_status st = sync_and_check(h);
    if (st != LB_OK) return st;
    prof.resize((size_t)h->n_cells * h->ny);
    wall.resize((size_t)h->n_cells * 2);
    CK(h, cudaMemcpy(prof.data(), h->acc_prof, sizeof(double) * prof.size(), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(wall.data(), h->acc_wall, sizeof(double) * wall.size(), cudaMemcpyDeviceToHost));
    return LB_OK;
}

lb_status lb_shear_stress(lb_handle* h, double* sigma_xy, double* shear_rate, double* shear_bulk)
{
    Trace trace("lb_shear_stress");
    if (!h) return LB_ERR_INVALID;
    if (!sigma_xy || !shear_rate) return fail(h, LB_ERR_INVALID, "lb_shear_stress: outputs are NULL");
    if (h->slab)
        return fail(h, LB_ERR_UNSUPPORTED, "lb_shear_stress: a slab holds part of the cell (combine lb_get_profile "
                    "and lb_wall_momentum over the slabs)");
    std::vector<double> prof, wall;
    lb_status st = read_acc(h, prof, wall);
    if (st != LB_OK) return st;
    const double ns = (double)h->n_samples, nx = h->nx;
    const int ny = h->ny, lo = ny / 4, hi = ny - ny / 4;
    for (int c = 0; c < h->n_cells; ++c) {
        if (h->n_samples == 0) {
            sigma_xy[c] = shear_rate[c] = NAN;
            if (shear_bulk) shear_bulk[c] = NAN;
            continue;
        }
        sigma_xy[c] = 0.5 * (wall[c * 2 + 0] - wall[c * 2 + 1]) / (nx * ns);
        const double* p = prof.data() + (size_t)c * ny;
        shear_rate[c] = (p[ny - 1] - p[0]) / (nx * ns) / (ny - 1);
        if (shear_bulk) {
            double ym = 0.5 * (lo + hi - 1), num = 0.0, den = 0.0;
            for (int y = lo; y < hi; ++y) {
                num += (y - ym) * (p[y] / (nx * ns));
                den += (y - ym) * (y - ym);
            }
            shear_bulk[c] = num / den;
        }
    }
    return LB_OK;
}

lb_status lb_get_profile(lb_handle* h, double* ubar, long long* n_samples)
{
    if (!h) return LB_ERR_INVALID;
    if (!ubar) return fail(h, LB_ERR_INVALID, "lb_get_profile: ubar is NULL");
    std::vector<double> prof, wall;
    lb_status st = read_acc(h, prof, wall);
    if (st != LB_OK) return st;
    const double d = (double)h->nx * (double)h->n_samples;
    for (size_t k = 0; k < prof.size(); ++k) ubar[k] = h->n_samples ? prof[k] / d : NAN;
    if (n_samples) *n_samples = h->n_samples;
    return LB_OK;
}

lb_status lb_get_fields(lb_handle* h, double* rho_a, double* rho_b, double* ux, double* uy)
{
    Trace trace("lb_get_fields");
    if (!h) return LB_ERR_INVALID;
    if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_get_fields: no state loaded");
    CK(h, cudaSetDevice(h->device));
    const size_t n = (size_t)h->nx * h->ny;
    if (!h->staging) CK(h, cudaMalloc(&h->staging, sizeof(double) * 4 * n * h->n_cells));
    CK(h, with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        return launch_fields<T>((const T*)fview(h, h->cur), h->staging, h->g, h->d_cells, h->d_err, h->stream);
    }));
    h->launches += 1;
    double* dst[4] = {rho_a, rho_b, ux, uy};
    for (int a = 0; a < 4; ++a)
        if (dst[a])
            CK(h, cudaMemcpy2DAsync(dst[a], n * sizeof(double), h->staging + a * n, 4 * n * sizeof(double),
                                    n * sizeof(double), h->n_cells, cudaMemcpyDeviceToHost, h->stream));
    return sync_and_check(h);
}

lb_status lb_reductions(lb_handle* h, double* mass_ab, double* momentum_xy)
{
    Trace trace("lb_reductions");
    if (!h) return LB_ERR_INVALID;
    if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_reductions: no state loaded");
    CK(h, cudaSetDevice(h->device));
    CK(h, with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        return launch_state_sums<T>((const T*)fview(h, h->cur), h->g, h->d_cells, h->red_part, h->red_out, h->d_err,
                                    h->stream);
    }));
    h->launches += 2;
    std::vector<double> o((size_t)h->n_cells * 4);
    CK(h, cudaMemcpyAsync(o.data(), h->red_out, sizeof(double) * o.size(), cudaMemcpyDeviceToHost, h->stream));
    lb_status st = sync_and_check(h);
    if (st != LB_OK) return st;
    for (int c = 0; c < h->n_cells; ++c) {
        if (mass_ab) {
            mass_ab[2 * c] = o[4 * c];
            mass_ab[2 * c + 1] = o[4 * c + 1];
        }
        if (momentum_xy) {
            momentum_xy[2 * c] = o[4 * c + 2];
            momentum_xy[2 * c + 1] = o[4 * c + 3];
        }
    }
    return LB_OK;
}

lb_status lb_set_kernel(lb_handle* h, lb_kernel kernel, int tile_x, int tile_y)
{
    if (!h) return LB_ERR_INVALID;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    return select_kernel(h, kernel, tile_x, tile_y);
}

lb_status lb_get_kernel(const lb_handle* h, lb_kernel* kernel, int* tile_x, int* tile_y)
{
    if (!h) return LB_ERR_INVALID;
    if (kernel) *kernel = h->kernel;
    if (tile_x) *tile_x = h->tile_x;
    if (tile_y) *tile_y = h->tile_y;
    return LB_OK;
}

lb_status lb_launch_shape(const lb_handle* h, int* ctas, int* ctas_sampled, int* threads, int* smem_bytes)
{
    if (!h) return LB_ERR_INVALID;
    if (h->kernel != LB_KERNEL_TILED || !h->plan) return LB_ERR_UNSUPPORTED;
    tiled_launch_shape(h->plan, ctas, ctas_sampled, threads, smem_bytes);
    return LB_OK;
}

lb_status lb_autotune(lb_handle* h, const char* cache_path)
{
    Trace trace("lb_autotune");
    if (!h) return LB_ERR_INVALID;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    char devname[256] = "";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) snprintf(devname, sizeof devname, "%s", prop.name);
    for (char* c = devname; *c; ++c)
        if (*c == ' ') *c = '_';
    char key[512];
    snprintf(key, sizeof key, "%s nx=%d ny=%d cells=%d prec=%d bc=%d%s", devname, h->nx, h->ny, h->n_cells,
             (int)h->prec, h->bc, h->slab ? " slab" : "");
    if (cache_path) {
        FILE* fp = fopen(cache_path, "r");
        if (fp) {
            char line[768];
            while (fgets(line, sizeof line, fp)) {
                int k = -1, tx = 0, ty = 0;
                char* bar = strchr(line, '|');
                if (!bar) continue;
                *bar = 0;
                if (strcmp(line, key) == 0 && sscanf(bar + 1, "%d %d %d", &k, &tx, &ty) == 3) {
                    fclose(fp);
                    return select_kernel(h, (lb_kernel)k, tx, ty);
                }
            }
            fclose(fp);
        }
    }
    // candidates: generic, and every supported tile
    std::vector<std::tuple<int, int, int>> cand;
    cand.emplace_back((int)LB_KERNEL_GENERIC, 0, 0);
    const int txs[] = {32, 64, 128, 256};
    const int tys[] = {0, 16, 32, 64};  // 0: segment height from the fill model
    for (int tx : txs)
        for (int ty : tys)
            if (tiled_supported(h->gbuf, h->elem, tx, ty)) cand.emplace_back((int)LB_KERNEL_TILED, tx, ty);
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    float best = 1e30f;
    std::tuple<int, int, int> best_c = cand[0];
    const int reps = 6;
    for (auto& c : cand) {
        if (select_kernel(h, (lb_kernel)std::get<0>(c), std::get<1>(c), std::get<2>(c)) != LB_OK) continue;
        int nl = 0;
        // trial steps read the current buffer and write the other one, without
        // swapping, so the state is unchanged
        bool ok = true;
        for (int r = 0; r < 2 && ok; ++r) ok = enqueue_one_step(h, h->cur, false, &nl) == cudaSuccess;
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && ok; ++r) ok = enqueue_one_step(h, h->cur, false, &nl) == cudaSuccess;
        cudaEventRecord(e1, h->stream);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        h->launches += nl;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lb_status st = select_kernel(h, (lb_kernel)std::get<0>(best_c), std::get<1>(best_c), std::get<2>(best_c));
    if (st != LB_OK) return st;
    if (cache_path) {
        FILE* fp = fopen(cache_path, "a");
        if (fp) {
            fprintf(fp, "%s|%d %d %d %.6f\n", key, std::get<0>(best_c), std::get<1>(best_c), std::get<2>(best_c),
                    best / reps);
            fclose(fp);
        }
    }
    return LB_OK;
}

lb_status lb_test_inject(lb_handle* h, int fault)
{
    if (!h) return LB_ERR_INVALID;
    if (fault < 0 || fault > 2) return fail(h, LB_ERR_INVALID, "lb_test_inject: unknown fault %d", fault);
    if (fault == 1 && h->kernel != LB_KERNEL_TILED)
        return fail(h, LB_ERR_UNSUPPORTED, "lb_test_inject: a stalled copy needs the tiled kernel");
    h->inject = fault;
    return LB_OK;
}

lb_status lb_sync(lb_handle* h)
{
    if (!h) return LB_ERR_INVALID;
    return sync_and_check(h);
}

long long lb_steps_done(const lb_handle* h) { return h ? h->t : 0; }

void* lb_stream(const lb_handle* h) { return h ? (void*)h->stream : nullptr; }

long long lb_kernel_launches(const lb_handle* h) { return h ? h->launches : 0; }

const char* lb_last_error(const lb_handle* h)
{
    if (!h) return g_create_msg[0] ? g_create_msg : g_null_msg;
    return h->last_error.c_str();
}

void lb_destroy(lb_handle* h) { release(h); }


lb_status lb_save(lb_handle* h, const char* path)
{
    Trace trace("lb_save");
    if (!h) return LB_ERR_INVALID;
    if (!path) return fail(h, LB_ERR_INVALID, "lb_save: path is NULL");
    if (h->slab) return fail(h, LB_ERR_UNSUPPORTED, "lb_save: not available for a slab");
    if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_save: no state loaded");
    lb_status st = sync_and_check(h);
    if (st != LB_OK) return st;
    std::vector<double> prof, wall;
    st = read_acc(h, prof, wall);
    if (st != LB_OK) return st;
    File out;
    out.f = fopen(path, "wb");
    if (!out.f) return fail(h, LB_ERR_INVALID, "lb_save: cannot open %s for writing", path);
    CkptHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, kMagic, 8);
    hd.version = 3;
    hd.header_bytes = sizeof hd;
    hd.n_cells = h->n_cells;
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.bc = h->bc;
    hd.prec = (int32_t)h->prec;
    hd.elem = h->elem;
    hd.t = h->t;
    hd.start = h->start;
    hd.every = h->every;
    hd.n_samples = h->n_samples;
    bool ok = fwrite(&hd, sizeof hd, 1, out.f) == 1;  // rewritten with the checksum at the end
    Fnv sum;
    uint64_t bytes = 0;
    auto put = [&](const void* p, size_t n) {
        if (!ok) return;
        ok = fwrite(p, 1, n, out.f) == n;
        sum.add(p, n);
        bytes += n;
    };
    for (int c = 0; c < h->n_cells; ++c) {
        double v[kCellDoubles];
        cell_to_doubles(h->cells[c], v);
        put(v, sizeof v);
    }
    put(prof.data(), sizeof(double) * prof.size());
    put(wall.data(), sizeof(double) * wall.size());
    const size_t row = (size_t)h->nx * h->elem, cell_bytes = row * 18 * h->ny;
    std::vector<unsigned char> buf(cell_bytes);
    for (int c = 0; c < h->n_cells && ok; ++c) {
        const unsigned char* src = (const unsigned char*)h->f[h->cur] + (size_t)c * h->g.cellstride * h->elem;
        CK(h, cudaMemcpy2D(buf.data(), row, src, (size_t)h->g.pitch * h->elem, row, (size_t)18 * h->ny,
                           cudaMemcpyDeviceToHost));
        put(buf.data(), cell_bytes);
    }
    hd.payload_bytes = bytes;
    hd.checksum = sum.h;
    if (ok) ok = fseek(out.f, 0, SEEK_SET) == 0 && fwrite(&hd, sizeof hd, 1, out.f) == 1;
    if (ok) ok = fclose(out.f) == 0;
    out.f = nullptr;
    if (!ok) return fail(h, LB_ERR_INVALID, "lb_save: writing %s failed", path);
    return LB_OK;
}

lb_status lb_load(lb_handle* h, const char* path)
{
    Trace trace("lb_load");
    if (!h) return LB_ERR_INVALID;
    if (!path) return fail(h, LB_ERR_INVALID, "lb_load: path is NULL");
    if (h->slab) return fail(h, LB_ERR_UNSUPPORTED, "lb_load: not available for a slab");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    h->batch_pending = false;
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return fail(h, LB_ERR_INVALID, "lb_load: cannot open %s", path);
    CkptHeader hd;
    if (fread(&hd, sizeof hd, 1, in.f) != 1 || memcmp(hd.magic, kMagic, 8) != 0)
        return fail(h, LB_ERR_INVALID, "lb_load: %s is not a checkpoint", path);
    if (hd.version < 1 || hd.version > 3 || hd.header_bytes != sizeof hd)
        return fail(h, LB_ERR_INVALID, "lb_load: checkpoint version %u not supported", hd.version);
    if (hd.n_cells != h->n_cells || hd.nx != h->nx || hd.ny != h->ny || hd.bc != h->bc ||
        hd.prec != (int32_t)h->prec || hd.elem != h->elem)
        return fail(h, LB_ERR_INVALID,
                    "lb_load: checkpoint holds %d cells of %dx%d (bc %d, precision %d), the handle %d of %dx%d "
                    "(bc %d, precision %d)", hd.n_cells, hd.nx, hd.ny, hd.bc, hd.prec, h->n_cells, h->nx, h->ny,
                    h->bc, (int)h->prec);
    if (hd.t < 0 || hd.start < 0 || hd.every < 0 || hd.n_samples < 0)
        return fail(h, LB_ERR_INVALID, "lb_load: negative counters in %s", path);
    // from here on the handle's state is being replaced: it only counts as
    // loaded once everything has been read and checked
    h->initialised = false;
    Fnv sum;
    uint64_t bytes = 0;
    bool ok = true;
    auto get = [&](void* p, size_t n) {
        if (!ok) return;
        ok = fread(p, 1, n, in.f) == n;
        if (ok) {
            sum.add(p, n);
            bytes += n;
        }
    };
    std::vector<lb_cell_params> cells(h->n_cells);
    bool cells_ok = true;
    const int per_cell = hd.version == 1 ? 14 : hd.version == 2 ? 15 : kCellDoubles;
    for (int c = 0; c < h->n_cells; ++c) {
        double v[kCellDoubles] = {};
        get(v, sizeof(double) * per_cell);
        if (ok) cells_ok = cell_from_doubles(v, &cells[c]) && cells_ok;
    }
    std::vector<double> prof((size_t)h->n_cells * h->ny), wall((size_t)h->n_cells * 2);
    get(prof.data(), sizeof(double) * prof.size());
    get(wall.data(), sizeof(double) * wall.size());
    const size_t row = (size_t)h->nx * h->elem, cell_bytes = row * 18 * h->ny;
    std::vector<unsigned char> buf(cell_bytes);
    for (int c = 0; c < h->n_cells && ok; ++c) {
        get(buf.data(), cell_bytes);
        if (!ok) break;
        unsigned char* dst = (unsigned char*)h->f[0] + (size_t)c * h->g.cellstride * h->elem;
        CK(h, cudaMemcpy2D(dst, (size_t)h->g.pitch * h->elem, buf.data(), row, row, (size_t)18 * h->ny,
                           cudaMemcpyHostToDevice));
    }
    unsigned char extra;
    if (!ok || bytes != hd.payload_bytes || fread(&extra, 1, 1, in.f) == 1)
        return fail(h, LB_ERR_INVALID, "lb_load: %s is truncated or has a different size than recorded", path);
    if (sum.h != hd.checksum) return fail(h, LB_ERR_INVALID, "lb_load: checksum mismatch in %s", path);
    char why[256] = "lattice size or boundary differs from the handle's";
    if (!cells_ok || !cells_valid(cells.data(), h->n_cells, why, sizeof why) || cells[0].nx != h->nx ||
        cells[0].ny != h->ny || cells[0].bc != h->bc)
        return fail(h, LB_ERR_INVALID, "lb_load: cell parameters in %s: %s", path, cells_ok ? why : "malformed");
    std::vector<CellDev> dc(h->n_cells);
    for (int c = 0; c < h->n_cells; ++c) dc[c] = to_dev(cells[c]);
    CK(h, cudaMemcpy(h->d_cells, dc.data(), sizeof(CellDev) * h->n_cells, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->acc_prof, prof.data(), sizeof(double) * prof.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->acc_wall, wall.data(), sizeof(double) * wall.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->d_err, 0, sizeof(unsigned)));
    h->h_err[0] = 0;
    h->cells = cells;
    if (h->plan) tiled_set_collision(h->plan, collision_kind(h->cells));
    free_graphs(h);  // captured launches may name the other kernel family
    h->cur = 0;
    h->t = hd.t;
    h->start = hd.start;
    h->every = hd.every;
    h->n_samples = hd.n_samples;
    h->faulted = false;
    h->initialised = true;
    return LB_OK;
}

// ------------------------------------------------------------------ slabs --
// Rows and planes of a slab message.  Buffer rows of a slab of `rows` own rows:
// 0, 1 ghost rows below | 2 .. rows+1 own rows | rows+2, rows+3 ghost rows above.
static bool slab_message(const lb_handle* h, int part, bool put, SlabMsg* m)
{
    const int rows = h->ny;
    const int up[6] = {2, 5, 6, 11, 14, 15}, down[6] = {4, 7, 8, 13, 16, 17};  // c_y = +1 / -1, both species
    switch (part) {
    case LB_SLAB_EDGE_LO:  // send: own rows 0, 1; receive: the ghost rows below
    case LB_SLAB_EDGE_HI:  // send: own rows rows-2, rows-1; receive: the ghost rows above
        m->n_planes = 18;
        for (int q = 0; q < 18; ++q) m->planes[q] = q;
        m->nrows = 2;
        m->row0 = part == LB_SLAB_EDGE_LO ? (put ? 0 : 2) : (put ? rows + 2 : rows);
        return true;
    case LB_SLAB_FLOW_LO:  // send: what streamed down out of the slab; receive: what streamed up into row 0
    case LB_SLAB_FLOW_HI:  // send: what streamed up out of the slab; receive: what streamed down into the last row
    {
        const bool lo = part == LB_SLAB_FLOW_LO;
        const int* q = (lo == put) ? up : down;
        m->n_planes = 6;
        for (int k = 0; k < 6; ++k) m->planes[k] = q[k];
        m->nrows = 1;
        m->row0 = lo ? (put ? 2 : 1) : (put ? rows + 1 : rows + 2);
        return true;
    }
    default:
        return false;
    }
}

static size_t slab_message_size(const lb_handle* h, const SlabMsg& m)
{
    return (size_t)h->n_cells * m.n_planes * m.nrows * h->nx * h->elem;
}

static lb_status slab_transfer(lb_handle* h, lb_slab_part part, void* buf, bool put, const char* name)
{
    if (!h) return LB_ERR_INVALID;
    if (!h->slab) return fail(h, LB_ERR_UNSUPPORTED, "%s: the handle holds whole cells, not a slab", name);
    if (!buf) return fail(h, LB_ERR_INVALID, "%s: the message buffer is NULL", name);
    SlabMsg m{};
    if (!slab_message(h, (int)part, put, &m)) return fail(h, LB_ERR_INVALID, "%s: unknown part %d", name, (int)part);
    if (!h->initialised) return fail(h, LB_ERR_STATE, "%s: no state loaded", name);
    CK(h, cudaSetDevice(h->device));
    char why[256];
    if (!device_buffer_ok(buf, slab_message_size(h, m), h->device, "message", why, sizeof why))
        return fail(h, LB_ERR_INVALID, "%s: %s", name, why);
    CK(h, with_type(h, [&](auto* tp) {
        using T = std::remove_pointer_t<decltype(tp)>;
        return launch_slab_msg<T>((T*)h->f[h->cur], (T*)buf, h->gbuf, m, !put, h->stream);
    }));
    h->launches += 1;
    return LB_OK;
}

lb_status lb_slab_info(const lb_handle* h, int* y0, int* rows, int* ny_global)
{
    if (!h) return LB_ERR_INVALID;
    if (y0) *y0 = h->rm.y0g;
    if (rows) *rows = h->ny;
    if (ny_global) *ny_global = h->rm.nyg;
    return h->slab ? LB_OK : LB_ERR_UNSUPPORTED;
}

lb_status lb_slab_message_bytes(const lb_handle* h, lb_slab_part part, size_t* bytes)
{
    if (!h || !bytes) return LB_ERR_INVALID;
    SlabMsg m{};
    if (!h->slab || !slab_message(h, (int)part, false, &m)) return h->slab ? LB_ERR_INVALID : LB_ERR_UNSUPPORTED;
    *bytes = slab_message_size(h, m);
    return LB_OK;
}

lb_status lb_slab_get(lb_handle* h, lb_slab_part part, void* dst)
{
    Trace trace("lb_slab_get");
    return slab_transfer(h, part, dst, false, "lb_slab_get");
}

lb_status lb_slab_put(lb_handle* h, lb_slab_part part, const void* src)
{
    Trace trace("lb_slab_put");
    return slab_transfer(h, part, const_cast<void*>(src), true, "lb_slab_put");
}

lb_status lb_wall_momentum(lb_handle* h, double* sums, long long* n_samples)
{
    if (!h) return LB_ERR_INVALID;
    if (!sums) return fail(h, LB_ERR_INVALID, "lb_wall_momentum: sums is NULL");
    std::vector<double> prof, wall;
    lb_status st = read_acc(h, prof, wall);
    if (st != LB_OK) return st;
    for (size_t k = 0; k < wall.size(); ++k) sums[k] = wall[k];
    if (n_samples) *n_samples = h->n_samples;
    return LB_OK;
}

}  // extern "C"
