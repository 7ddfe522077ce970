// Generic kernel family: any lattice size, every storage precision.
//   moments_psi : rho_s = sum_i f_is and psi_s(rho_s) into an auxiliary field
//   fused_generic: interaction forces (Eq. (FFF)) from that field, shifted BGK
//                  collision (Eq. (be)) and push streaming with the boundaries,
//                  plus, on sampled steps, FP64 partial sums of the observables.
// One thread per site.  The tiled family (lb_tiled.cu) is the fast path; this
// one serves shapes the tiled kernel does not take and is the second opinion in
// tests.
#include "lb_internal.h"

namespace lbhb {

template <class T>
__global__ void __launch_bounds__(256) moments_psi_kernel(const T* __restrict__ f, Geom g,
                                                          const CellDev* __restrict__ cells,
                                                          typename Store<T>::C* __restrict__ aux)
{
    using C = typename Store<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int cell = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const ParamSet<C>& p = params<C>(cells[cell]);
    const long long n = (long long)g.nx * g.ny;
    C* a = aux + (long long)cell * 4 * n + (long long)y * g.nx + x;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        C r = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C sh = Store<T>::shifted ? pop_shift<C>(i, p, s) : C(0);
            r += Store<T>::ld(f, fidx(g, cell, s * 9 + i, y, x), sh);
        }
        a[s * n] = r;
        a[(2 + s) * n] = psi_of(r, p.rho0, p.inv_rho0);
    }
}

template <class T, bool SAMPLE>
__global__ void __launch_bounds__(256) fused_generic_kernel(const T* __restrict__ fin, T* __restrict__ fout, Geom g,
                                                            int bc, const CellDev* __restrict__ cells,
                                                            const typename Store<T>::C* __restrict__ aux,
                                                            double* __restrict__ prof_part,
                                                            double* __restrict__ wall_part,
                                                            unsigned* __restrict__ err)
{
    using C = typename Store<T>::C;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int cell = blockIdx.z;
    const bool active = x < g.nx && y < g.ny;
    const ParamSet<C>& p = params<C>(cells[cell]);
    const long long n = (long long)g.nx * g.ny;
    const C* rho_f = aux + (long long)cell * 4 * n;
    double uphys = 0.0, dpx_site = 0.0;
    bool bad = false;  // watchdog: non-finite or non-positive density at this site

    if (active) {
        C f[2][9];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const C sh = Store<T>::shifted ? pop_shift<C>(i, p, s) : C(0);
                f[s][i] = Store<T>::ld(fin, fidx(g, cell, s * 9 + i, y, x), sh);
            }
        const long long k0 = (long long)y * g.nx + x;
        C rho[2] = {rho_f[k0], rho_f[n + k0]};
        C psi[2] = {rho_f[2 * n + k0], rho_f[3 * n + k0]};
        Sums<C> sm[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            C dpsi[12], drho[4];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const int xp = wrap_x(x + hs_dx(k), g.nx), xm = wrap_x(x - hs_dx(k), g.nx);
                const int yp = stencil_row(y + hs_dy(k), g.ny, bc), ym = stencil_row(y - hs_dy(k), g.ny, bc);
                const long long kp = (long long)yp * g.nx + xp, km = (long long)ym * g.nx + xm;
                dpsi[k] = rho_f[(2 + s) * n + kp] - rho_f[(2 + s) * n + km];
                if (k < 4) drho[k] = rho_f[(1 - s) * n + kp] - rho_f[(1 - s) * n + km];
            }
            sm[s] = stencil_sums<C>(dpsi, drho);
        }
        Collided<C> c;
        collide_site<C>(f, rho, psi, sm, p, body_force_x<C>(p, y), c);

        const C u_top = p.u_wall, u_bot = -p.u_wall;
        Dither dz;  // stochastic rounding stream of this site (dithered storage only)
        if constexpr (Store<T>::dithered)
            dz.seed(((uint32_t)cell * 0x9E3779B1u) ^ ((uint32_t)y << 15) ^ ((uint32_t)x << 1),
                    __float_as_uint(rho[0]) ^ (__float_as_uint(rho[1]) * 0x85EBCA6Bu));
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int yd = y + q_cy(i);
                const C sh = Store<T>::shifted ? pop_shift<C>(i, p, s) : C(0);
                if (bc == 1 && (yd < 0 || yd >= g.ny)) {
                    C dpx;
                    const C back = bounce<C>(i, c.fs[s][i], rho[s], yd < 0 ? u_bot : u_top, &dpx);
                    const C sho = Store<T>::shifted ? pop_shift<C>(q_opp(i), p, s) : C(0);
                    Store<T>::st(fout, fidx(g, cell, s * 9 + q_opp(i), y, x), back, sho, dz);
                    dpx_site += (double)dpx;
                } else {
                    const int xd = wrap_x(x + q_cx(i), g.nx);
                    const int ydd = yd < 0 ? yd + g.ny : (yd >= g.ny ? yd - g.ny : yd);
                    Store<T>::st(fout, fidx(g, cell, s * 9 + i, ydd, xd), c.fs[s][i], sh, dz);
                }
            }
        const C rt = rho[0] + rho[1];
        bad = !(rt > C(0)) || !isfinite((double)rho[0]) || !isfinite((double)rho[1]);
        if (SAMPLE) {
            // force-corrected velocity (j + F/2)/rho
            const C jx = mom_x<C>(f[0]) + mom_x<C>(f[1]);
            uphys = (double)((jx + C(0.5) * c.Fx) / rt);
        }
    }
    // every step, sampled or not: one flag per warp into the error word
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_NONFINITE);
    if (SAMPLE) {
        // FP64 warp sums: one warp = 32 consecutive columns of one row.
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            uphys += __shfl_down_sync(0xffffffffu, uphys, o);
            dpx_site += __shfl_down_sync(0xffffffffu, dpx_site, o);
        }
        if (threadIdx.x == 0 && y < g.ny) {
            const int nbx = gridDim.x;
            prof_part[((long long)cell * nbx + blockIdx.x) * g.ny + y] = uphys;
            if (bc == 1 && (y == 0 || y == g.ny - 1))
                wall_part[((long long)cell * nbx + blockIdx.x) * 2 + (y == 0 ? 1 : 0)] = dpx_site;
        }
    }
}

template <class T>
cudaError_t launch_generic_step(const T* fin, T* fout, const Geom& g, int bc, const CellDev* cells,
                                void* aux, bool sample, double* prof_part, double* wall_part,
                                unsigned* err, cudaStream_t st, int* n_launches)
{
    using C = typename Store<T>::C;
    dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.n_cells);
    moments_psi_kernel<T><<<grd, blk, 0, st>>>(fin, g, cells, (C*)aux);
    if (sample)
        fused_generic_kernel<T, true><<<grd, blk, 0, st>>>(fin, fout, g, bc, cells, (const C*)aux, prof_part,
                                                          wall_part, err);
    else
        fused_generic_kernel<T, false><<<grd, blk, 0, st>>>(fin, fout, g, bc, cells, (const C*)aux, prof_part,
                                                           wall_part, err);
    *n_launches += 2;
    return cudaGetLastError();
}

int generic_partials_nbx(const Geom& g) { return (g.nx + 31) / 32; }

template cudaError_t launch_generic_step<float>(const float*, float*, const Geom&, int, const CellDev*, void*, bool,
                                                double*, double*, unsigned*, cudaStream_t, int*);
template cudaError_t launch_generic_step<double>(const double*, double*, const Geom&, int, const CellDev*, void*,
                                                 bool, double*, double*, unsigned*, cudaStream_t, int*);
template cudaError_t launch_generic_step<__half>(const __half*, __half*, const Geom&, int, const CellDev*, void*,
                                                 bool, double*, double*, unsigned*, cudaStream_t, int*);
template cudaError_t launch_generic_step<half_sr>(const half_sr*, half_sr*, const Geom&, int, const CellDev*, void*,
                                                  bool, double*, double*, unsigned*, cudaStream_t, int*);

}  // namespace lbhb
