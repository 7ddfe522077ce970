// Non-hot-path kernels: initial equilibrium, population import/export, field
// readout, FP64 reductions of the state and of the sampled observables.
#include "lb_internal.h"

namespace lbhb {

// f_is = f^eq_is(rho_s, u): w_i rho_s (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u^2), cs^2 = 1/3,
// evaluated in the compute type of the storage (FP32 for FP32 and FP16 storage:
// the FP64 pipe would make this initialisation ten times slower than its
// memory traffic), the +-c pairs together as in the collision.
// src: device float64 [cell][4][ny][nx] = rho_A, rho_B, u_x, u_y.
template <class T>
__global__ void equilibrium_kernel(const double* __restrict__ src, T* __restrict__ f, Geom g,
                                   const CellDev* __restrict__ cells)
{
    using C = typename Store<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, cell = blockIdx.z;
    if (x >= g.nx) return;
    const long long n = (long long)g.nx * g.ny, k = (long long)y * g.nx + x;
    const double* s0 = src + (long long)cell * 4 * n;
    const C ux = C(s0[2 * n + k]), uy = C(s0[3 * n + k]);
    const C base = C(1) - C(1.5) * (ux * ux + uy * uy);
    const C cu[4] = {ux, uy, ux + uy, uy - ux};  // c.u for i = 1, 2, 5, 6
    const int lo[4] = {1, 2, 5, 6}, hi[4] = {3, 4, 7, 8};
    const ParamSet<C>& p = params<C>(cells[cell]);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const C r = C(s0[s * n + k]);
        const C sh0 = Store<T>::shifted ? pop_shift<C>(0, p, s) : C(0);
        Store<T>::st(f, fidx(g, cell, s * 9, y, x), C(q_w(0)) * r * base, sh0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C wr = C(q_w(lo[q])) * r;
            const C a = wr * (base + C(4.5) * cu[q] * cu[q]), b = (C(3) * wr) * cu[q];
            const C shi = Store<T>::shifted ? pop_shift<C>(lo[q], p, s) : C(0);
            const C sho = Store<T>::shifted ? pop_shift<C>(hi[q], p, s) : C(0);
            Store<T>::st(f, fidx(g, cell, s * 9 + lo[q], y, x), a + b, shi);
            Store<T>::st(f, fidx(g, cell, s * 9 + hi[q], y, x), a - b, sho);
        }
    }
}

// Storage <-> dense float64 [cell][18][ny][nx].
template <class T>
__global__ void export_kernel(const T* __restrict__ f, double* __restrict__ dst, Geom g,
                              const CellDev* __restrict__ cells)
{
    using C = typename Store<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, cq = blockIdx.z;
    if (x >= g.nx) return;
    const int cell = cq / 18, q = cq % 18, s = q / 9, i = q % 9;
    const C sh = Store<T>::shifted ? pop_shift<C>(i, params<C>(cells[cell]), s) : C(0);
    dst[(((long long)cell * 18 + q) * g.ny + y) * g.nx + x] = (double)Store<T>::ld(f, fidx(g, cell, q, y, x), sh);
}

template <class T>
__global__ void import_kernel(const double* __restrict__ src, T* __restrict__ f, Geom g,
                              const CellDev* __restrict__ cells)
{
    using C = typename Store<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, cq = blockIdx.z;
    if (x >= g.nx) return;
    const int cell = cq / 18, q = cq % 18, s = q / 9, i = q % 9;
    const C sh = Store<T>::shifted ? pop_shift<C>(i, params<C>(cells[cell]), s) : C(0);
    Store<T>::st(f, fidx(g, cell, q, y, x), C(src[(((long long)cell * 18 + q) * g.ny + y) * g.nx + x]), sh);
}

// Per-site rho_A, rho_B, and the paper's u = j / rho into dense float64
// [cell][4][ny][nx]; flags non-finite or non-positive densities.
template <class T>
__global__ void fields_kernel(const T* __restrict__ f, double* __restrict__ dst, Geom g,
                              const CellDev* __restrict__ cells, unsigned* __restrict__ err)
{
    using C = typename Store<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, cell = blockIdx.z;
    if (x >= g.nx) return;
    double rho[2], jx = 0.0, jy = 0.0;
    for (int s = 0; s < 2; ++s) {
        C v[9];
        C r = C(0);
        for (int i = 0; i < 9; ++i) {
            const C sh = Store<T>::shifted ? pop_shift<C>(i, params<C>(cells[cell]), s) : C(0);
            v[i] = Store<T>::ld(f, fidx(g, cell, s * 9 + i, y, x), sh);
            r += v[i];
        }
        rho[s] = (double)r;
        jx += (double)((v[1] - v[3]) + (v[5] - v[7]) + (v[8] - v[6]));
        jy += (double)((v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]));
    }
    const long long n = (long long)g.nx * g.ny, k = (long long)y * g.nx + x;
    double* d = dst + (long long)cell * 4 * n;
    const double rt = rho[0] + rho[1];
    d[k] = rho[0];
    d[n + k] = rho[1];
    d[2 * n + k] = jx / rt;
    d[3 * n + k] = jy / rt;
    if (!(rt > 0.0) || !isfinite(rho[0]) || !isfinite(rho[1])) atomicOr(err, ERR_NONFINITE);
}

// FP64 state sums, pass 1: block b of cell c sums sites [b*chunk, (b+1)*chunk)
// into part[c][b][4] = (sum rho_A, sum rho_B, sum j_x, sum j_y), by a fixed-shape
// tree, so results are reproducible run to run.
constexpr int RED_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(RED_THREADS) state_sums_kernel(const T* __restrict__ f, Geom g,
                                                                 const CellDev* __restrict__ cells,
                                                                 long long chunk, double* __restrict__ part,
                                                                 unsigned* __restrict__ err)
{
    using C = typename Store<T>::C;
    const int cell = blockIdx.y;
    const long long n = (long long)g.nx * g.ny;
    const long long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long k = lo + threadIdx.x; k < hi; k += RED_THREADS) {
        const int y = (int)(k / g.nx), x = (int)(k % g.nx);
        double rt = 0.0;
        for (int s = 0; s < 2; ++s) {
            C v[9];
            C r = C(0);
            for (int i = 0; i < 9; ++i) {
                const C sh = Store<T>::shifted ? pop_shift<C>(i, params<C>(cells[cell]), s) : C(0);
                v[i] = Store<T>::ld(f, fidx(g, cell, s * 9 + i, y, x), sh);
                r += v[i];
            }
            acc[s] += (double)r;
            rt += (double)r;
            bad |= !isfinite((double)r);
            acc[2] += (double)((v[1] - v[3]) + (v[5] - v[7]) + (v[8] - v[6]));
            acc[3] += (double)((v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]));
        }
        bad |= !(rt > 0.0);
    }
    if (bad) atomicOr(err, ERR_NONFINITE);
    __shared__ double sh[4][RED_THREADS];
    for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] = acc[a];
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[((long long)cell * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

// Pass 2: out[c][a] = sum over blocks b (in order) of part[c][b][a].
__global__ void state_sums_finish(const double* __restrict__ part, int nblk, double* __restrict__ out)
{
    const int cell = blockIdx.x, a = threadIdx.x;
    if (a >= 4) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((long long)cell * nblk + b) * 4 + a];
    out[cell * 4 + a] = s;
}

// Folds the partials of one sampled step into the time averages:
// acc_prof[c][y] += sum_b prof_part[c][b][y];  acc_wall[c][w] += sum_b wall_part[c][b][w].
// One warp per (cell, block of 32 rows), spread over the whole GPU.
__global__ void accumulate_kernel(const double* __restrict__ prof_part, const double* __restrict__ wall_part,
                                  int nbx, int ny, int bc, double* __restrict__ acc_prof,
                                  double* __restrict__ acc_wall)
{
    const int cell = blockIdx.x;
    const int y = blockIdx.y * 32 + threadIdx.x;
    if (y < ny) {
        double s = 0.0;
        for (int b = 0; b < nbx; ++b) s += prof_part[((long long)cell * nbx + b) * ny + y];
        acc_prof[(long long)cell * ny + y] += s;
    }
    if (bc == 1 && blockIdx.y == 0 && threadIdx.x < 2) {
        double s = 0.0;
        for (int b = 0; b < nbx; ++b) s += wall_part[((long long)cell * nbx + b) * 2 + threadIdx.x];
        acc_wall[cell * 2 + threadIdx.x] += s;
    }
}

// Slab messages: `planes` of rows [row0, row0 + nrows) of the population
// buffer of every cell, packed as [cell][plane k][row r][x] (dense in x), in
// the storage format (no conversion).
template <class T>
__global__ void slab_msg_kernel(T* __restrict__ f, T* __restrict__ msg, Geom g, SlabMsg m, int pack)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.nx) return;
    const int k = blockIdx.y / m.nrows, r = blockIdx.y % m.nrows, cell = blockIdx.z;
    const long long km = (((long long)cell * m.n_planes + k) * m.nrows + r) * g.nx + x;
    const long long kf = fidx(g, cell, m.planes[k], m.row0 + r, x);
    if (pack)
        msg[km] = f[kf];
    else
        f[kf] = msg[km];
}

// ------------------------------------------------------------ launchers --
template <class T>
cudaError_t launch_slab_msg(T* f, T* msg, const Geom& g, const SlabMsg& m, bool pack, cudaStream_t st)
{
    dim3 blk(128), grd((g.nx + 127) / 128, m.n_planes * m.nrows, g.n_cells);
    slab_msg_kernel<T><<<grd, blk, 0, st>>>(f, msg, g, m, pack ? 1 : 0);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_equilibrium(const double* src, T* f, const Geom& g, const CellDev* cells, cudaStream_t st)
{
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.n_cells);
    equilibrium_kernel<T><<<grd, blk, 0, st>>>(src, f, g, cells);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_export(const T* f, double* dst, const Geom& g, const CellDev* cells, cudaStream_t st)
{
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.n_cells * 18);
    export_kernel<T><<<grd, blk, 0, st>>>(f, dst, g, cells);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_import(const double* src, T* f, const Geom& g, const CellDev* cells, cudaStream_t st)
{
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.n_cells * 18);
    import_kernel<T><<<grd, blk, 0, st>>>(src, f, g, cells);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_fields(const T* f, double* dst, const Geom& g, const CellDev* cells, unsigned* err,
                          cudaStream_t st)
{
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny, g.n_cells);
    fields_kernel<T><<<grd, blk, 0, st>>>(f, dst, g, cells, err);
    return cudaGetLastError();
}

int state_sums_blocks(const Geom& g)
{
    const long long n = (long long)g.nx * g.ny;
    long long nb = (n + 8191) / 8192;
    return (int)(nb < 1 ? 1 : (nb > 1024 ? 1024 : nb));
}

template <class T>
cudaError_t launch_state_sums(const T* f, const Geom& g, const CellDev* cells, double* part, double* out,
                              unsigned* err, cudaStream_t st)
{
    const int nb = state_sums_blocks(g);
    const long long n = (long long)g.nx * g.ny;
    const long long chunk = (n + nb - 1) / nb;
    state_sums_kernel<T><<<dim3(nb, g.n_cells), RED_THREADS, 0, st>>>(f, g, cells, chunk, part, err);
    state_sums_finish<<<g.n_cells, 32, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const double* prof_part, const double* wall_part, int nbx, int ny, int bc,
                              int n_cells, double* acc_prof, double* acc_wall, cudaStream_t st)
{
    accumulate_kernel<<<dim3(n_cells, (ny + 31) / 32), 32, 0, st>>>(prof_part, wall_part, nbx, ny, bc, acc_prof,
                                                                      acc_wall);
    return cudaGetLastError();
}

#define LBHB_INST(T)                                                                                        \
    template cudaError_t launch_equilibrium<T>(const double*, T*, const Geom&, const CellDev*, cudaStream_t); \
    template cudaError_t launch_export<T>(const T*, double*, const Geom&, const CellDev*, cudaStream_t);      \
    template cudaError_t launch_import<T>(const double*, T*, const Geom&, const CellDev*, cudaStream_t);      \
    template cudaError_t launch_fields<T>(const T*, double*, const Geom&, const CellDev*, unsigned*,          \
                                          cudaStream_t);                                                    \
    template cudaError_t launch_state_sums<T>(const T*, const Geom&, const CellDev*, double*, double*,       \
                                              unsigned*, cudaStream_t);                                     \
    template cudaError_t launch_slab_msg<T>(T*, T*, const Geom&, const SlabMsg&, bool, cudaStream_t);
LBHB_INST(float)
LBHB_INST(double)
LBHB_INST(__half)
LBHB_INST(half_sr)

}  // namespace lbhb
