// Tiled single-pass kernel family: the whole time step (moments, pseudopotential,
// 25-point forces of Eq. (FFF), shifted BGK collision of Eq. (be), streaming)
// in one pass over the populations.
//
// Work item = one column strip of TX sites x one segment of TY rows of one cell.
// A CTA has TX column threads (one species and two adjacent columns each: lanes
// 0-15 of a warp species A, 16-31 species B of the same 32 columns) and one
// service warp (TMA issue, halo columns of psi/rho, row sums of sampled steps).
// It walks its segment row by row:
//   * TMA (cp.async.bulk.tensor, 4-D map [cell][q][y][x]) brings whole rows of all
//     18 populations into a ring of D shared-memory slots, several rows ahead,
//     each slot completing on its own mbarrier; a row is TX main columns plus
//     16-byte halo boxes on both sides (periodic wrap in x by coordinates);
//   * when row y+2 lands, its rho_s and psi_s (for the TX columns and 2 halo
//     columns per side) go into a 6-row ring, so rows y-2..y+2 of psi/rho are
//     on chip when row y is collided: the 25-point stencil reads shared memory;
//   * row y is collided from its populations still in the slot ring and pushed
//     to the other ping-pong buffer with plain coalesced stores (x-shifted by
//     -1/0/+1 element), bounce-back rows handled in place; with FP16 storage the
//     stores round to nearest or stochastically (Store<T>, Dither).
// HBM traffic per site update is one read and one write of the 18 populations;
// halo rows/columns are re-read by neighbouring work items (mostly from L2).
// The grid is persistent (CTAs loop over work items).  Every mbarrier wait is
// bounded: on timeout the CTA records ERR_TIMEOUT, drains its copies in flight
// (also bounded) and leaves.
#include <cudaTypedefs.h>

#include <algorithm>
#include <limits>
#include <type_traits>

#include "lb_internal.h"
#include "lbhb.h"
#include "tma.cuh"

namespace lbhb {

constexpr int RING = 6;  // psi/rho rows on chip: 5 read by a collision + 1 being written

__host__ __device__ constexpr int al128(int b) { return (b + 127) / 128 * 128; }

struct SlotGeom {
    int main_b, halo_b, main_al, halo_al, slot_b, tx_bytes, halo;
};

__host__ __device__ inline SlotGeom slot_geom(int tx, int elem)
{
    SlotGeom s;
    s.halo = 16 / elem;
    s.main_b = 18 * tx * elem;
    s.halo_b = 18 * s.halo * elem;
    s.main_al = al128(s.main_b);
    s.halo_al = al128(s.halo_b);
    s.slot_b = s.main_al + 2 * s.halo_al;
    s.tx_bytes = s.main_b + 2 * s.halo_b;
    return s;
}

struct TiledPlan {
    Geom g;     // the whole population buffer (for a slab: its own rows and two ghost rows each side)
    RowMap rm;  // the rows a step updates
    int elem, bc, tx, ty, depth;
    int n_strips, n_seg;
    int grid[3][2];  // persistent CTAs: [kernel family FAM_*][plain 0 / sampled 1]
    size_t smem;
    CUtensorMap tm_main[2], tm_halo[2];
    void* f[2];
    uint32_t skip_row = ~0u;  // failure injection for the next launch (tests)
    int collision = TILED_BGK_ONE_TIME;  // the cells' collision (tiled_set_collision)
};

// Row-slot ring depth: about three rows in flight beyond the three in use.
// FP64 rows are consumed at the FP64 pipe's pace (a seventh of the FP32 rate),
// so one row in flight covers the memory latency, and the smaller ring lets two
// CTAs share an SM.
__host__ __device__ constexpr int ring_depth(int tx, int elem)
{
    return elem == 8 ? 4 : (6 * al128(18 * tx * elem) + 12 * al128(18 * (16 / elem) * elem) <= 96 * 1024) ? 6 : 5;
}
// Words between the species-A and species-B psi/rho rings, chosen so that a
// half-warp reading A and the other half reading B hit disjoint banks.
__host__ __device__ constexpr int ring_species_stride(int tx)
{
    return RING * (tx + 4) + ((16 - (RING * (tx + 4)) % 32) + 32) % 32;
}

// Two adjacent columns of one species per thread: vector (8-byte for FP32)
// shared-memory accesses and two independent sites per thread.
template <class T> struct Vec2;
template <> struct Vec2<float> {
    __device__ static void ld(const float* p, float& a, float& b)
    {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static void st(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
};
template <> struct Vec2<double> {
    __device__ static void ld(const double* p, double& a, double& b)
    {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static void st(double* p, double a, double b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }
};
template <> struct Vec2<__half> {
    __device__ static void ld(const __half* p, float& a, float& b)
    {
        const __half2 v = *reinterpret_cast<const __half2*>(p);
        a = __low2float(v);
        b = __high2float(v);
    }
    // FP16 storage of shifted values: the caller subtracts the shift
    __device__ static void st(__half* p, float a, float b) { *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b); }
};
// stochastically rounded FP16: loads as for __half (the caller unscales),
// stores with the thread's dither stream
template <> struct Vec2<half_sr> {
    __device__ static void ld(const half_sr* p, float& a, float& b)
    {
        const __half2 v = *reinterpret_cast<const __half2*>(p);
        a = __low2float(v);
        b = __high2float(v);
    }
    __device__ static void st(half_sr* p, float a, float b, Dither& d)
    {
        const __half lo = half_sr_round(a, d), hi = half_sr_round(b, d);
        *reinterpret_cast<__half2*>(p) = __halves2half2(lo, hi);
    }
};
// paired and single stores of values already in the stored representation,
// dithered where the storage asks for it
template <class T, class C>
__device__ inline void st_pair(T* p, C a, C b, Dither& d)
{
    if constexpr (Store<T>::dithered)
        Vec2<T>::st(p, a, b, d);
    else
        Vec2<T>::st(p, a, b);
}
template <class T, class C>
__device__ inline void st_one(T* p, C v, Dither& d)
{
    if constexpr (std::is_same<T, half_sr>::value)
        p->h = half_sr_round(v, d);
    else if constexpr (std::is_same<T, __half>::value)
        *p = __float2half_rn(v);
    else
        *p = v;
}

// Element CI (0..5) of a window row of six columns held as three lane pairs.
template <int CI, class C>
__device__ __forceinline__ C win_at(const P2<C> (&row)[3])
{
    return (CI & 1) ? row[CI >> 1].b() : row[CI >> 1].a();
}

// g(r + c) - g(r - c) of Eq. (FFF) for both sites of a thread, c = (DX, DY):
// site o sits at column 2 + o of window row MID.  Pairs at an even column
// offset are the stored pairs (one packed subtraction); odd offsets straddle
// two pairs (two scalar subtractions).
template <int DX, int DY, int MID, int NR, class C>
__device__ __forceinline__ P2<C> pair_diff(const P2<C> (&w)[NR][3])
{
    constexpr int cp = 2 + DX, cm = 2 - DX;
    if constexpr ((DX & 1) == 0)
        return w[MID + DY][cp / 2] - w[MID - DY][cm / 2];
    else
        return P2<C>(win_at<cp>(w[MID + DY]) - win_at<cm>(w[MID - DY]),
                     win_at<cp + 1>(w[MID + DY]) - win_at<cm + 1>(w[MID - DY]));
}

// The half-stencil differences of psi (window rows k-2..k+2) and of the partner
// density rho_s' (rows k-1..k+1, belt 1 only), in the order of hs_dx / hs_dy.
template <class C>
__device__ __forceinline__ void window_diffs(const P2<C> (&v)[5][3], const P2<C> (&e)[3][3], P2<C> d[12],
                                             P2<C> de[4])
{
    d[0] = pair_diff<hs_dx(0), hs_dy(0), 2>(v);
    d[1] = pair_diff<hs_dx(1), hs_dy(1), 2>(v);
    d[2] = pair_diff<hs_dx(2), hs_dy(2), 2>(v);
    d[3] = pair_diff<hs_dx(3), hs_dy(3), 2>(v);
    d[4] = pair_diff<hs_dx(4), hs_dy(4), 2>(v);
    d[5] = pair_diff<hs_dx(5), hs_dy(5), 2>(v);
    d[6] = pair_diff<hs_dx(6), hs_dy(6), 2>(v);
    d[7] = pair_diff<hs_dx(7), hs_dy(7), 2>(v);
    d[8] = pair_diff<hs_dx(8), hs_dy(8), 2>(v);
    d[9] = pair_diff<hs_dx(9), hs_dy(9), 2>(v);
    d[10] = pair_diff<hs_dx(10), hs_dy(10), 2>(v);
    d[11] = pair_diff<hs_dx(11), hs_dy(11), 2>(v);
    de[0] = pair_diff<hs_dx(0), hs_dy(0), 1>(e);
    de[1] = pair_diff<hs_dx(1), hs_dy(1), 1>(e);
    de[2] = pair_diff<hs_dx(2), hs_dy(2), 1>(e);
    de[3] = pair_diff<hs_dx(3), hs_dy(3), 1>(e);
}

// Threads per CTA: a thread per (species, column pair), TX threads, plus one
// service warp that issues the TMA copies and computes the four halo columns
// of psi/rho, so the column warps all do the same work between two barriers.
__host__ __device__ constexpr int tiled_threads(int tx) { return tx + 32; }

// Dynamic shared memory of a CTA: row slots, psi/rho rings, mbarriers, and two
// rows of per-site profile values (sampled steps).
__host__ __device__ constexpr int tiled_smem_bytes(int tx, int elem)
{
    return ring_depth(tx, elem) * (al128(18 * tx * elem) + 2 * al128(18 * (16 / elem) * elem)) +
           4 * ring_species_stride(tx) * (elem == 8 ? 8 : 4) + ring_depth(tx, elem) * 8 + 2 * tx * (elem == 8 ? 8 : 4);
}
// CTAs of a plain step per SM that shared memory admits (228 KB per SM, 1 KB of
// it reserved per CTA), at most 4: the register budget the compiler is held to,
// so that registers do not admit fewer.  Sampled steps (a tenth of the launches,
// with more live values) are held to at most 3.
__host__ __device__ constexpr int tiled_min_ctas(int tx, int elem)
{
    return 233472 / (tiled_smem_bytes(tx, elem) + 1024) < 1   ? 1
         : 233472 / (tiled_smem_bytes(tx, elem) + 1024) > 4 ? 4
                                                             : 233472 / (tiled_smem_bytes(tx, elem) + 1024);
}

// Service warp, sampled steps: the sums of u_x over each 32-column group of one
// row of a strip (ub: TX values), one FP64 partial per group as the column warps
// would have written it.  Lane l takes NW = TX/32 consecutive columns of group
// l / (32/NW), then a segmented warp sum; FP32 values are carried as an
// unevaluated (hi, lo) pair (error-free two-sum), ~2^-48 relative.  Not inlined,
// so its registers do not add to the column warps' in the hot loop.
template <class C, int TX>
__device__ __noinline__ void profile_row_sums(const C* ub, int lane, double* __restrict__ prof_part, int cell,
                                              int nx, int nrows, int x0, int row)
{
    constexpr int NW = TX / 32, SEG = 32 / NW;
    const int grp = lane / SEG, t = lane % SEG;
    double part;
    if constexpr (sizeof(C) == 4) {
        float hi = ub[grp * 32 + t * NW], lo = 0.f;
#pragma unroll
        for (int q = 1; q < NW; ++q) {
            const float v = ub[grp * 32 + t * NW + q];
            const float sum = __fadd_rn(hi, v);
            const float bp = __fsub_rn(sum, hi);
            lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bp)), __fsub_rn(v, bp)));
            hi = sum;
        }
#pragma unroll
        for (int o = SEG / 2; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xffffffffu, hi, o, SEG);
            const float l2 = __shfl_down_sync(0xffffffffu, lo, o, SEG);
            const float sum = __fadd_rn(hi, h2);
            const float bp = __fsub_rn(sum, hi);
            const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bp)), __fsub_rn(h2, bp));
            hi = sum;
            lo = __fadd_rn(__fadd_rn(lo, l2), err);
        }
        part = (double)hi + (double)lo;
    } else {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < NW; ++q) v += ub[grp * 32 + t * NW + q];
#pragma unroll
        for (int o = SEG / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, SEG);
        part = v;
    }
    const int nbx = (nx + 31) / 32;  // 32-column groups of the lattice; a narrow last strip has fewer
    if (t == 0 && (x0 >> 5) + grp < nbx) prof_part[((long long)cell * nbx + (x0 >> 5) + grp) * nrows + row] = part;
}

// Kernel families (FAM):
//   FAM_FULL  every strip is TX columns wide (nx a multiple of TX) and every cell
//             has one relaxation time (BGK);
//   FAM_GEN   the last strip may be narrower (its extra columns masked) and the
//             species may relax with times of their own (BGK);
//   FAM_MRT   as FAM_GEN, with the multiple-relaxation-time collision.
constexpr int FAM_FULL = 0, FAM_GEN = 1, FAM_MRT = 2;
template <class T, int TX, bool SAMPLE, int FAM>
__global__ void __launch_bounds__(tiled_threads(TX),
                                  SAMPLE ? (tiled_min_ctas(TX, (int)sizeof(T)) < 3 ? tiled_min_ctas(TX, (int)sizeof(T)) : 3)
                                         : tiled_min_ctas(TX, (int)sizeof(T)))
    tiled_step_kernel(const __grid_constant__ CUtensorMap tm_main,
                                                            const __grid_constant__ CUtensorMap tm_halo,
                                                            T* __restrict__ fout, Geom g, int bc, RowMap rm,
                                                            int ty,
                                                            int n_strips, int n_seg,
                                                            const CellDev* __restrict__ cells,
                                                            double* __restrict__ prof_part,
                                                            double* __restrict__ wall_part,
                                                            unsigned* __restrict__ err, uint32_t skip_row_arg)
{
    using C = typename Store<T>::C;
    using V = P2<C>;  // a lane pair: one species at the thread's two sites
    constexpr bool FULL = FAM == FAM_FULL, MRT = FAM == FAM_MRT;
    // stored populations are scale * g (scale 1 except for the dithered FP16 storage)
    constexpr C scale = C(Store<T>::scale), inv_scale = C(1) / scale;
    constexpr int E = (int)sizeof(T);
    constexpr int H = 16 / E;            // halo columns per side brought by TMA
    constexpr int W = TX + 4;            // ring row: columns -2 .. TX+1
    constexpr int D = ring_depth(TX, E);
    constexpr int SS = ring_species_stride(TX);
    constexpr int MAIN_AL = al128(18 * TX * E);
    constexpr int HALO_AL = al128(18 * H * E);
    constexpr int SLOT = MAIN_AL + 2 * HALO_AL;
    constexpr uint32_t TX_BYTES = 18 * TX * E + 2 * 18 * H * E;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* fring = smem;
    C* psi_ring = reinterpret_cast<C*>(smem + D * SLOT);  // [species][RING][W] (stride SS per species)
    C* rho_ring = psi_ring + 2 * SS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(rho_ring + 2 * SS);
    // sampled steps: u_x of each site of the last two rows, summed by the service warp
    C* ubuf = reinterpret_cast<C*>(bars + D);

    constexpr int NW = TX / 32;               // column warps (32 columns x 2 species each)
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const bool svc = warp == NW;              // the service warp
    const bool producer = svc && lane == 0;   // issues the TMA copies
    // column warps: lanes 0-15 species A, 16-31 species B, columns c0 and c0+1;
    // service warp: lanes 0-3 species A, 4-7 species B of the halo columns
    const int sp = svc ? (lane >> 2) & 1 : lane >> 4;
    const int c0 = svc ? 0 : warp * 32 + 2 * (lane & 15);
    // a pipeline that timed out in an earlier launch of the same batch does not
    // run again (each later launch would otherwise wait out its own bound); the
    // decision is taken once per CTA, at the barrier that publishes the mbarriers
    bool stale = false;
    if (t == 0) {
        stale = (*reinterpret_cast<volatile unsigned*>(err) & ERR_TIMEOUT) != 0u;
        for (int d = 0; d < D; ++d) mbar_init(&bars[d], 1);
        fence_mbar_init();
        prefetch_tensormap(&tm_main);
        prefetch_tensormap(&tm_halo);
    }
    if (__syncthreads_or(stale)) return;

    // failure-injection hook (tests only): CTA 0 leaves the copy of its row
    // skip_row_arg unissued, so the waits for it run out; ~0u: none
    const uint32_t skip_row = blockIdx.x == 0 ? skip_row_arg : ~0u;
    const long long per_cell = (long long)n_strips * n_seg;
    const long long items = per_cell * g.n_cells;
    uint32_t nrow = 0;  // global index of row 0 of the current item (rows consumed before it)
    bool aborted = false;
    bool bad = false;  // watchdog: a non-finite or non-positive density seen in this item

    // Issue cursor (producer): the next row to load may belong to a later item
    // of this CTA, so the row pipeline does not drain between items.  Global
    // row n always lives in slot n % D with mbarrier phase (n / D) & 1.  The
    // geometry of the item being issued is cached (one division per item).
    long long iw = blockIdx.x;
    int ik = 0, icell = 0, ix0 = 0, iy0 = 0, iR = 0, ixl = 0, ixr = 0;
    uint32_t n_issued = 0;
    auto load_item = [&]() {
        if (iw >= items) return;
        icell = (int)(iw / per_cell);
        const int irem = (int)(iw - (long long)icell * per_cell);
        const int iseg = irem / n_strips;
        ix0 = (irem - iseg * n_strips) * TX;
        iy0 = rm.ylo + iseg * ty;
        iR = min(ty, rm.ylo + rm.nown - iy0) + 4;
        ixl = ix0 >= H ? ix0 - H : g.nx - H;
        ixr = ix0 + TX < g.nx ? ix0 + TX : 0;
    };
    if (producer) load_item();
    auto issue_upto = [&](uint32_t limit) {
        while (n_issued < limit && iw < items) {
            const int slot = (int)(n_issued % D);
            unsigned char* dst = fring + slot * SLOT;
            const int yp = stencil_load_row(iy0 - 2 + ik, g.ny, rm, bc);
            if (n_issued != skip_row) {
                mbar_arrive_expect_tx(&bars[slot], TX_BYTES);
                tma_load_4d(dst, &tm_main, ix0, yp, 0, icell, &bars[slot]);
                tma_load_4d(dst + MAIN_AL, &tm_halo, ixl, yp, 0, icell, &bars[slot]);
                tma_load_4d(dst + MAIN_AL + HALO_AL, &tm_halo, ixr, yp, 0, icell, &bars[slot]);
            }
            ++n_issued;
            if (++ik == iR) {
                ik = 0;
                iw += gridDim.x;
                load_item();
            }
        }
    };

    for (long long w = blockIdx.x; w < items && !aborted; w += gridDim.x) {
        const int cell = (int)(w / per_cell);
        const int rem = (int)(w % per_cell);
        const int seg = rem / n_strips, strip = rem % n_strips;
        const int x0 = strip * TX, y0 = rm.ylo + seg * ty;  // buffer row of the item's first row
        const int rows = min(ty, rm.ylo + rm.nown - y0);
        const int R = rows + 4;  // logical rows y0-2 .. y0+rows+1
        // per-cell parameters as scalars (no runtime-indexed arrays: they would
        // live in local memory)
        const ParamSet<C>& pg = params<C>(cells[cell]);
        ParamSet<C> p;
        p.rho0 = pg.rho0;
        p.inv_rho0 = pg.inv_rho0;
        p.gab_over_rho0 = pg.gab_over_rho0;
        p.u_wall = pg.u_wall;
        p.f0 = pg.f0;
        p.two_over_ny = pg.two_over_ny;
        // this lane's species relaxes with tau_s; mix weighs the partner species'
        // moments in the common velocity (1, and one_time, for one relaxation time)
        const C tau_s = FULL || !sp ? pg.tau : pg.tau_b, omega_s = FULL || !sp ? pg.omega : pg.omega_b;
        const C mix = FULL ? C(1) : (sp ? pg.mix[1] : pg.mix[0]);
        const bool one_time = FULL || pg.mix[0] == C(1);
        // tau = 1 for both species: f* = f^eq.  Uniform over the item, so both
        // half-warps take the same path (a cell with tau_A = 1 != tau_B runs the
        // general update in both)
        const bool unit_omega = FULL ? pg.omega == C(1) : (pg.omega == C(1) && pg.omega_b == C(1));
        // multiple-relaxation-time coefficients of this lane's species (mrt_delta)
        V mh[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) mh[q] = V(MRT ? (sp ? pg.mrt_h[1][q] : pg.mrt_h[0][q]) : C(0));
        // the same values as lane pairs
        const V ga = V(sp ? pg.g1[1] : pg.g1[0]), gr = V(sp ? pg.g2[1] : pg.g2[0]), gx = V(p.gab_over_rho0);
        const V tau2 = V(tau_s), ntau2 = V(-tau_s), omega2 = V(omega_s), mix2 = V(mix);
        const V rho0_2 = V(p.rho0), inv_rho0_2 = V(p.inv_rho0);
        const C rho_bar = sp ? pg.rho_bar[1] : pg.rho_bar[0];
        const V rho_bar2 = V(rho_bar);
        // columns of this strip inside the lattice (the last strip of a width that
        // is not a multiple of TX is narrower; the TMA box reads zeros beyond it)
        const int wv = FULL ? TX : min(TX, g.nx - x0);
        const bool act = FULL || c0 < wv;  // both columns of the pair (wv is even)
        // destination columns of the two sites x, x+1 shifted by -1/0/+1 (periodic)
        const int x = x0 + c0;
        const int col_m = x == 0 ? g.nx - 1 : x - 1, col_p2 = x + 2 == g.nx ? 0 : x + 2;
        T* const dst_s = fout + (long long)cell * g.cellstride + (long long)sp * 9 * g.plane;
        T* const dst_x = dst_s + x;  // column x, plane 0 of the species, row 0
        // warps holding column 0 or column nx - 1 wrap their x-shifted stores
        // periodically; the others store each direction's two sites at fixed
        // offsets from one address
        const bool xedge = (x0 == 0 && warp == 0) || (x0 + 32 * warp + 32 >= g.nx);

        // rings of the previous item are no longer read; the watchdog flags of its
        // rows are reported
        if (__syncthreads_or(bad) && t == 0) atomicOr(err, ERR_NONFINITE);
        bad = false;

        if (producer) issue_upto(nrow + D);  // rows of earlier items are all done
        auto wait_row = [&](int k) -> bool {
            const uint32_t n = nrow + (uint32_t)k;
            return mbar_wait_bounded(&bars[n % D], (n / D) & 1u);
        };
        // rho_s, psi_s of logical row k into ring row `ring_row` (own species,
        // own two columns; the service warp takes the halo columns)
        auto psi_stage_slot = [&](int slot, int ring_row) {
            const unsigned char* base = fring + slot * SLOT;
            const int ring = sp * SS + ring_row * W;
            if (!svc) {
                if (!act) return;  // its ring positions belong to the halo or to nobody
                const T* src = reinterpret_cast<const T*>(base) + sp * 9 * TX + c0;
                V r = Pair<T>::ld(src);
#pragma unroll
                for (int i = 1; i < 9; ++i) r = r + Pair<T>::ld(src + i * TX);
                if constexpr (Store<T>::shifted) {  // sum of the shifts w_i rho_bar is rho_bar
                    if constexpr (Store<T>::scale != 1)
                        r = vfma(r, V(inv_scale), rho_bar2);
                    else
                        r = r + rho_bar2;
                }
                Pair<C>::st(psi_ring + ring + c0 + 2, lane_psi(r, rho0_2, inv_rho0_2));
                Pair<C>::st(rho_ring + ring + c0 + 2, r);
            } else if (lane < 8) {
                // halo column h: 0,1 -> columns -2,-1 (left box); 2,3 -> TX, TX+1 (right box)
                const int h = lane & 3;
                const T* src = reinterpret_cast<const T*>(base + (h < 2 ? MAIN_AL : MAIN_AL + HALO_AL)) + sp * 9 * H +
                               (h < 2 ? H - 2 + h : h - 2);
                C acc = C(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) acc += to_c(src[i * H]);
                if (Store<T>::shifted) acc = acc * inv_scale + rho_bar;
                const int pos = h < 2 ? h : wv + h;
                psi_ring[ring + pos] = psi_of(acc, p.rho0, p.inv_rho0);
                rho_ring[ring + pos] = acc;
            }
        };

        bool ok = true;
        for (int k = 0; k < 4; ++k) {
            ok = wait_row(k) && ok;
            psi_stage_slot((int)((nrow + (uint32_t)k) % (uint32_t)D), k);
        }
        if constexpr (D < 5) {
            // a four-slot ring holds rows 0..3 only: rows 4 and 5 go into the slots of
            // rows 0 and 1 once every thread has staged those (the loop below waits
            // for row j + 4 before its own barrier)
            __syncthreads();
            if (producer) issue_upto(nrow + 2u + (uint32_t)D);
        }
        int r0 = 0;  // ring row of logical row j (rows j .. j+4 are read by the collision of row j+2)
        // slot and mbarrier phase of logical row j + 4 (global row nrow + j + 4),
        // advanced by one row per iteration instead of recomputed
        int s4 = (int)((nrow + 4u) % (uint32_t)D);
        uint32_t ph4 = ((nrow + 4u) / (uint32_t)D) & 1u;
        for (int j = 0; j < rows; ++j) {
            int rr[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) rr[d] = r0 + d >= RING ? r0 + d - RING : r0 + d;
            const int s2 = s4 >= 2 ? s4 - 2 : s4 + D - 2;  // slot of row j + 2
            ok = mbar_wait_bounded(&bars[s4], ph4) && ok;
            psi_stage_slot(s4, rr[4]);
            if (++s4 == D) {
                s4 = 0;
                ph4 ^= 1u;
            }
            r0 = rr[1];
            // barrier: psi/rho of row j+4 visible, collision of row j+1 finished
            // everywhere; it also tells every thread whether any wait ran out
            if (__syncthreads_or(ok ? 0 : 1)) {
                aborted = true;
                break;
            }
            // rows 0 .. j+1 of this item are done with their slots
            if (producer) issue_upto(nrow + (uint32_t)(j + 2 + D));
            if (svc) {
                if (SAMPLE && j > 0)  // its row finished before this barrier
                    profile_row_sums<C, TX>(ubuf + ((j - 1) & 1) * TX, lane, prof_part, cell, g.nx, rm.nown, x0,
                                            y0 + j - 1 - rm.ylo);
                continue;
            }
            // ---- collide logical row k = j + 2 (lattice row y), sites x and x+1
            const int y = y0 + j, gy = y - rm.ylo + rm.y0g;  // buffer row, row of the global cell
            const T* fm = reinterpret_cast<const T*>(fring + s2 * SLOT) + sp * 9 * TX + c0;
            // populations as stored: f for FP32/FP64, the shifted g for FP16; a
            // lane pair per direction (sites x, x+1)
            V f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = Pair<T>::ld(fm + i * TX);
            // psi window rows k-2..k+2 and rho_s' window rows k-1..k+1, columns
            // c0-2..c0+3 as three pairs; window column 2 + o is site o
            const C* ps = psi_ring + sp * SS + c0;  // ring column c0 + 2 + dx  <->  column c0 + dx
            const C* ro = rho_ring + (1 - sp) * SS + c0;
            V v[5][3], e[3][3];
#pragma unroll
            for (int d = 0; d < 5; ++d)
#pragma unroll
                for (int m = 0; m < 3; ++m) v[d][m] = Pair<C>::ld(ps + rr[d] * W + 2 * m);
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int m = 0; m < 3; ++m) e[d][m] = Pair<C>::ld(ro + rr[d + 1] * W + 2 * m);
            const V rho_s = Pair<C>::ld(rho_ring + sp * SS + rr[2] * W + c0 + 2);
            const V rho_p = e[1][1];  // the partner species' densities at the same two sites
            // pair differences d_q = psi(r + c_q) - psi(r - c_q) of both sites
            V dps[12], dro[4];
            window_diffs(v, e, dps, dro);
            const Sums<V> sm = stencil_sums<V>(dps, dro);
            const V jx_s = mom_x<V>(f), jy_s = mom_y<V>(f);
            const V jx_p(__shfl_xor_sync(0xffffffffu, jx_s.a(), 16), __shfl_xor_sync(0xffffffffu, jx_s.b(), 16));
            const V jy_p(__shfl_xor_sync(0xffffffffu, jy_s.a(), 16), __shfl_xor_sync(0xffffffffu, jy_s.b(), 16));
            // common velocity: (j_own + mix j_partner) / (rho_own + mix rho_partner)
            V jwx, jwy, rho_w;
            if constexpr (FULL) {  // one relaxation time: the barycentric velocity
                jwx = jx_s + jx_p;
                jwy = jy_s + jy_p;
                rho_w = rho_s + rho_p;
            } else {
                jwx = vfma(mix2, jx_p, jx_s);
                jwy = vfma(mix2, jy_p, jy_s);
                rho_w = vfma(mix2, rho_p, rho_s);
            }
            if constexpr (Store<T>::scale != 1) {
                jwx = jwx * V(inv_scale);
                jwy = jwy * V(inv_scale);
            }
            const V inv_rho = lane_rcp(rho_w);
            const V ux = jwx * inv_rho, uy = jwy * inv_rho;
            const C fx_body = body_force_x<C>(p, gy);
            const bool body_raw = !one_time && fx_body != C(0);  // the force needs the raw 1/rho
            const V rho_t = FULL ? rho_w : rho_s + rho_p;        // total density of each site
            V ax = V(fx_body) * inv_rho;
            if (body_raw) ax = V(fx_body) * lane_rcp(rho_t);
            // watchdog: a non-finite or non-positive total density anywhere in the
            // item is reported through the error word when the item ends
            if (act) bad |= !(rho_t.a() > C(0) && rho_t.a() <= std::numeric_limits<C>::max() && rho_t.b() > C(0) &&
                              rho_t.b() <= std::numeric_limits<C>::max());
            V fs[9], Fx, Fy;
            if constexpr (MRT && Store<T>::shifted) {
                collide_species_shifted<V, false, true>(f, rho_s, rho_bar2, v[2][1], ux, uy, ax, sm, ga, gr, gx,
                                                        tau2, ntau2, omega2, fs, &Fx, &Fy, V(scale), mh);
            } else if constexpr (MRT) {
                collide_species<V, false, true>(f, rho_s, v[2][1], ux, uy, ax, sm, ga, gr, gx, tau2, ntau2, omega2,
                                                fs, &Fx, &Fy, mh);
            } else if constexpr (Store<T>::shifted) {
                if (unit_omega)
                    collide_species_shifted<V, true>(f, rho_s, rho_bar2, v[2][1], ux, uy, ax, sm, ga, gr, gx, tau2,
                                                     ntau2, omega2, fs, &Fx, &Fy, V(scale));
                else
                    collide_species_shifted<V, false>(f, rho_s, rho_bar2, v[2][1], ux, uy, ax, sm, ga, gr, gx, tau2,
                                                      ntau2, omega2, fs, &Fx, &Fy, V(scale));
            } else {
                if (unit_omega)
                    collide_species<V, true>(f, rho_s, v[2][1], ux, uy, ax, sm, ga, gr, gx, tau2, ntau2, omega2, fs,
                                             &Fx, &Fy);
                else
                    collide_species<V, false>(f, rho_s, v[2][1], ux, uy, ax, sm, ga, gr, gx, tau2, ntau2, omega2, fs,
                                              &Fx, &Fy);
            }

            // stochastic rounding: one stream per thread and row, seeded from the
            // sites and their densities
            Dither dz;
            if constexpr (Store<T>::dithered)
                dz.seed(((uint32_t)cell * 0x9E3779B1u) ^ ((uint32_t)gy << 15) ^ ((uint32_t)x << 1) ^ (uint32_t)sp,
                        __float_as_uint(rho_s.a()) ^ (__float_as_uint(rho_s.b()) * 0x85EBCA6Bu));
            // push streaming; rows next to a Couette wall bounce back in place
            const bool wall_lo = bc == 1 && gy == 0, wall_hi = bc == 1 && gy == rm.nyg - 1;
            const int pl = (int)g.plane;  // < 2^31 / 18, checked on the host
            // destination rows y-1, y, y+1: periodic in a whole cell; a slab streams
            // into its ghost rows (the populations that leave it)
            const int row3[3] = {(!rm.slab && y == 0 ? g.ny - 1 : y - 1) * g.pitch, y * g.pitch,
                                 (!rm.slab && y == g.ny - 1 ? 0 : y + 1) * g.pitch};
            const int colA[3] = {col_m, x, x + 1};   // site x,   shifts -1, 0, +1
            const int colB[3] = {x, x + 1, col_p2};  // site x+1, shifts -1, 0, +1
            C dpx_site = C(0);
            if (act) {  // columns beyond the lattice store nothing
                if (!(wall_lo || wall_hi) && !xedge) {
                    // interior row (uniform over the CTA), away from the x edge (uniform
                    // over the warp): one address per direction, no wall tests
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int cy = q_cy(i), cx = q_cx(i);
                        T* const q = dst_x + (i * pl + row3[cy + 1]);
                        if (cx == 0) {
                            st_pair<T, C>(q, fs[i].a(), fs[i].b(), dz);
                        } else {
                            st_one<T, C>(q + cx, fs[i].a(), dz);
                            st_one<T, C>(q + cx + 1, fs[i].b(), dz);
                        }
                    }
                } else if (!(wall_lo || wall_hi)) {
                    // interior row on a warp at the x edge: periodic columns
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int cy = q_cy(i), cx = q_cx(i);
                        if (cx == 0) {
                            st_pair<T, C>(dst_s + i * pl + row3[cy + 1] + x, fs[i].a(), fs[i].b(), dz);
                        } else {
                            st_one<T, C>(dst_s + i * pl + row3[cy + 1] + colA[cx + 1], fs[i].a(), dz);
                            st_one<T, C>(dst_s + i * pl + row3[cy + 1] + colB[cx + 1], fs[i].b(), dz);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int cy = q_cy(i), cx = q_cx(i);
                        const bool into_wall = (cy < 0 && wall_lo) || (cy > 0 && wall_hi);
                        if (into_wall) {
                            C dpa, dpb;
                            const C uw = cy < 0 ? -p.u_wall : p.u_wall;
                            // bounce in the f representation (for shifted storage the shift
                            // is put back first; opposite directions carry equal weights,
                            // so the same shift is removed again)
                            const C sh = Store<T>::shifted ? C(q_w(i)) * rho_bar : C(0);
                            const C ba = bounce<C>(i, fs[i].a() * inv_scale + sh, rho_s.a(), uw, &dpa);
                            const C bb = bounce<C>(i, fs[i].b() * inv_scale + sh, rho_s.b(), uw, &dpb);
                            st_pair<T, C>(dst_s + q_opp(i) * pl + row3[1] + x, (ba - sh) * scale, (bb - sh) * scale, dz);
                            dpx_site += dpa + dpb;
                        } else if (cx == 0) {
                            st_pair<T, C>(dst_s + i * pl + row3[cy + 1] + x, fs[i].a(), fs[i].b(), dz);
                        } else {
                            st_one<T, C>(dst_s + i * pl + row3[cy + 1] + colA[cx + 1], fs[i].a(), dz);
                            st_one<T, C>(dst_s + i * pl + row3[cy + 1] + colB[cx + 1], fs[i].b(), dz);
                        }
                    }
                }
            }
            if (SAMPLE) {
                // force-corrected velocity (j + F/2)/rho of the observables, from the
                // raw barycentric momentum and density
                V jxo = jwx, inv_r = inv_rho;
                if (!one_time) {
                    jxo = jx_s + jx_p;
                    if constexpr (Store<T>::scale != 1) jxo = jxo * V(inv_scale);
                    inv_r = lane_rcp(rho_t);
                }
                // one site per lane: species-A lanes take column x, species-B
                // lanes column x+1; each lane sends its partner the force the
                // partner's site needs, so one shuffle gives F_x of both species
                const C fx_partner = __shfl_xor_sync(0xffffffffu, sp ? Fx.a() : Fx.b(), 16);
                const C Fx_t = (sp ? Fx.b() : Fx.a()) + fx_partner;
                const C up = ((sp ? jxo.b() : jxo.a()) + C(0.5) * Fx_t) * (sp ? inv_r.b() : inv_r.a());
                // the row sums of u_x are the service warp's (svc_profile, after the
                // next barrier): sums carried as an unevaluated pair (error-free
                // two-sum), then added in FP64, ~2^-48 relative
                ubuf[(j & 1) * TX + c0 + sp] = act ? up : C(0);
                if (wall_lo || wall_hi) {
                    const double wsum = warp_sum_compensated2(dpx_site, C(0));
                    const int nbx = (g.nx + 31) / 32, wg = (x0 >> 5) + warp;
                    if (lane == 0 && wg < nbx) wall_part[((long long)cell * nbx + wg) * 2 + (wall_lo ? 1 : 0)] = wsum;
                }
            }
        }
        if (SAMPLE && !aborted) {
            __syncthreads();  // the last row's u_x values are in place
            if (svc)
                profile_row_sums<C, TX>(ubuf + ((rows - 1) & 1) * TX, lane, prof_part, cell, g.nx, rm.nown, x0,
                                        y0 + rows - 1 - rm.ylo);
        }
        if (aborted) {
            if (producer) {
                atomicOr(err, ERR_TIMEOUT);
                // drain the copies still in flight before shared memory is released
                for (uint32_t n = nrow; n < n_issued; ++n)
                    if (n != skip_row) mbar_wait_bounded(&bars[n % D], (n / D) & 1u, 500000000ull);
            }
            __syncthreads();
            break;
        }
        nrow += (uint32_t)R;
    }
    if (__syncthreads_or(bad) && t == 0) atomicOr(err, ERR_NONFINITE);
}

// ------------------------------------------------------------- host side --
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static int depth_for(int tx, int elem) { return ring_depth(tx, elem); }

static size_t smem_bytes(int tx, int elem, int depth)
{
    const SlotGeom sg = slot_geom(tx, elem);
    const int cb = elem == 8 ? 8 : 4;
    // slots, psi/rho rings, mbarriers, and two rows of per-site profile values
    const size_t b = (size_t)depth * sg.slot_b + (size_t)4 * ring_species_stride(tx) * cb + (size_t)depth * 8 +
                     (size_t)2 * tx * cb;
    return b;
}
static_assert(tiled_smem_bytes(128, 4) == 74032, "shared memory of the FP32 128-column tile");

// Segment height from a fill model: work items = strips x segments x cells run
// on `slots` persistent CTAs, each item costing about (rows + 6) row-times
// (4 halo rows plus pipeline effects); pick the height with the least
// rounds x cost, so the last round of items is not mostly empty.
static int pick_segment_rows(const Geom& g, int nrows, int tile_x, long long slots)
{
    const long long strips = g.nx / tile_x;
    int best = 32;
    double best_cost = 1e300;
    for (int ty = 8; ty <= 256 && ty <= nrows; ++ty) {
        const long long items = strips * g.n_cells * ((nrows + ty - 1) / ty);
        const long long rounds = (items + slots - 1) / slots;
        const int rows = std::min(ty, nrows);
        const double cost = (double)rounds * (rows + 6);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = ty;
        }
    }
    return best;
}

bool tiled_supported(const Geom& g, int elem, int tile_x, int tile_y)
{
    if (tile_x != 32 && tile_x != 64 && tile_x != 128 && tile_x != 256) return false;
    // tile_y 0: chosen by the fill model.  nx need not be a multiple of the tile
    // (the last strip is narrower) but must be even (column pairs) and its rows
    // 16-byte multiples (TMA strides and halo coordinates).
    if (tile_y < 0 || g.nx % 2 != 0 || g.ny < 5) return false;
    if (g.nx < tile_x || (g.nx * elem) % 16 != 0) return false;
    if (18 * g.plane >= (1LL << 31)) return false;  // 32-bit element offsets inside a cell
    if (smem_bytes(tile_x, elem, depth_for(tile_x, elem)) > 227 * 1024) return false;
    return encode_fn() != nullptr;
}

int tiled_partials_nbx(const Geom& g, int) { return (g.nx + 31) / 32; }

template <class T, int TX, int FAM>
static const void* kernel_ptr(bool sample)
{
    return sample ? reinterpret_cast<const void*>(&tiled_step_kernel<T, TX, true, FAM>)
                  : reinterpret_cast<const void*>(&tiled_step_kernel<T, TX, false, FAM>);
}

template <class T, int TX>
static const void* kernel_ptr(bool sample, int fam)
{
    return fam == FAM_FULL ? kernel_ptr<T, TX, FAM_FULL>(sample)
         : fam == FAM_GEN  ? kernel_ptr<T, TX, FAM_GEN>(sample)
                           : kernel_ptr<T, TX, FAM_MRT>(sample);
}

template <class T>
static const void* pick(int tx, bool sample, int fam)
{
    switch (tx) {
    case 32: return kernel_ptr<T, 32>(sample, fam);
    case 64: return kernel_ptr<T, 64>(sample, fam);
    case 128: return kernel_ptr<T, 128>(sample, fam);
    default: return kernel_ptr<T, 256>(sample, fam);
    }
}

static const void* pick_any(int prec, int tx, bool sample, int fam)
{
    switch (prec) {
    case LB_FP32: return pick<float>(tx, sample, fam);
    case LB_FP64: return pick<double>(tx, sample, fam);
    case LB_FP16_SHIFTED_SR: return pick<half_sr>(tx, sample, fam);
    default: return pick<__half>(tx, sample, fam);
    }
}

// The family a launch runs: the full-width one when the strips are whole and
// every cell has one relaxation time and BGK, else the general or MRT one.
static int launch_family(const TiledPlan* p)
{
    if (p->collision == TILED_MRT) return FAM_MRT;
    return p->g.nx % p->tx == 0 && p->collision == TILED_BGK_ONE_TIME ? FAM_FULL : FAM_GEN;
}

static bool encode(CUtensorMap* m, void* base, const Geom& g, int elem, int box_x)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const CUtensorMapDataType dt = elem == 4   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 18, (cuuint64_t)g.n_cells};
    cuuint64_t strides[3] = {(cuuint64_t)g.pitch * elem, (cuuint64_t)g.plane * elem,
                             (cuuint64_t)g.cellstride * elem};
    cuuint32_t box[4] = {(cuuint32_t)box_x, 1, 18, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, dt, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

TiledPlan* tiled_create(const Geom& g, const RowMap& rm, int prec, int elem, int bc, void* f0, void* f1, int tile_x,
                        int tile_y, const char** err_msg)
{
    if (!tiled_supported(g, elem, tile_x, tile_y)) {
        if (err_msg) *err_msg = "shape/tile not supported by the tiled kernel";
        return nullptr;
    }
    TiledPlan* p = new TiledPlan();
    p->g = g;
    p->rm = rm;
    p->elem = elem;
    p->bc = bc;
    p->tx = tile_x;
    p->ty = tile_y;
    p->depth = depth_for(tile_x, elem);
    p->n_strips = (g.nx + tile_x - 1) / tile_x;
    p->smem = smem_bytes(tile_x, elem, p->depth);
    p->f[0] = f0;
    p->f[1] = f1;
    const int halo = 16 / elem;
    for (int b = 0; b < 2; ++b)
        if (!encode(&p->tm_main[b], b ? f1 : f0, g, elem, tile_x) || !encode(&p->tm_halo[b], b ? f1 : f0, g, elem, halo)) {
            if (err_msg) *err_msg = "cuTensorMapEncodeTiled failed";
            delete p;
            return nullptr;
        }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // occupancy of each kernel: the full-width family (nx a multiple of the tile,
    // one relaxation time), the general one and the MRT one, each plain and
    // sampled; which family runs depends on the cells' collision, which lb_load
    // may change, so all are prepared.  Plain and sampled launches of a family
    // share the work items (the segment height) but each runs as many persistent
    // CTAs as fit (the sampled variant holds more registers)
    const bool full_ok = g.nx % tile_x == 0;
    int occ[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int s = 0; s < 6; ++s) {
        const int fam = s >> 1, smp = s & 1;
        if (fam == FAM_FULL && !full_ok) continue;
        const void* k = pick_any(prec, tile_x, smp != 0, fam);
        // the whole unified L1/shared array as shared memory: the CTAs' rings
        // are what sets how many fit on an SM
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem) != cudaSuccess ||
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) {
            cudaGetLastError();
            if (err_msg) *err_msg = "cudaFuncSetAttribute(max dynamic smem) failed";
            delete p;
            return nullptr;
        }
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, tiled_threads(tile_x), p->smem) != cudaSuccess ||
            o < 1) {
            cudaGetLastError();
            if (err_msg) *err_msg = "tiled kernel does not fit on an SM";
            delete p;
            return nullptr;
        }
        occ[fam][smp] = o;
    }
    // segment height for the plain kernel of the family that will run most
    const long long slots = (long long)sms * occ[full_ok ? 0 : 1][0];
    if (p->ty <= 0) p->ty = pick_segment_rows(g, rm.nown, tile_x, slots);
    p->n_seg = (rm.nown + p->ty - 1) / p->ty;
    const long long items = (long long)p->n_strips * p->n_seg * g.n_cells;
    for (int fam = 0; fam < 3; ++fam)
        for (int smp = 0; smp < 2; ++smp)
            p->grid[fam][smp] = occ[fam][smp] > 0 ? (int)std::min(items, (long long)sms * occ[fam][smp]) : 0;
    return p;
}

void tiled_destroy(TiledPlan* p) { delete p; }

void tiled_inject_skip(TiledPlan* p, uint32_t row) { p->skip_row = row; }

void tiled_set_collision(TiledPlan* p, int collision) { p->collision = collision; }

void tiled_tiles(const TiledPlan* p, int* tx, int* ty)
{
    *tx = p->tx;
    *ty = p->ty;
}

void tiled_launch_shape(const TiledPlan* p, int* grid_plain, int* grid_sampled, int* threads, int* smem)
{
    const int fam = launch_family(p);
    if (grid_plain) *grid_plain = p->grid[fam][0];
    if (grid_sampled) *grid_sampled = p->grid[fam][1];
    if (threads) *threads = tiled_threads(p->tx);
    if (smem) *smem = (int)p->smem;
}

template <class T>
cudaError_t launch_tiled_step(TiledPlan* p, int src, const CellDev* cells, bool sample, double* prof_part,
                              double* wall_part, unsigned* err, cudaStream_t st, int* n_launches)
{
    T* dst = reinterpret_cast<T*>(p->f[1 - src]);
    const int fam = launch_family(p);
    const void* k = pick<T>(p->tx, sample, fam);
    Geom g = p->g;
    RowMap rm = p->rm;
    int bc = p->bc, ty = p->ty, ns = p->n_strips, nseg = p->n_seg;
    uint32_t skip = p->skip_row;
    p->skip_row = ~0u;  // one launch only
    void* args[] = {(void*)&p->tm_main[src], (void*)&p->tm_halo[src], (void*)&dst, (void*)&g, (void*)&bc,
                    (void*)&rm, (void*)&ty, (void*)&ns, (void*)&nseg, (void*)&cells, (void*)&prof_part,
                    (void*)&wall_part, (void*)&err, (void*)&skip};
    cudaError_t e = cudaLaunchKernel(k, dim3(p->grid[fam][sample ? 1 : 0]), dim3(tiled_threads(p->tx)), args,
                                     p->smem, st);
    *n_launches += 1;
    return e;
}

template cudaError_t launch_tiled_step<float>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                              cudaStream_t, int*);
template cudaError_t launch_tiled_step<double>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                               cudaStream_t, int*);
template cudaError_t launch_tiled_step<__half>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                               cudaStream_t, int*);
template cudaError_t launch_tiled_step<half_sr>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                                cudaStream_t, int*);

}  // namespace lbhb
