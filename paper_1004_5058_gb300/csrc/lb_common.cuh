// Shared device-side definitions of the CUDA path: lattice tables, per-cell
// parameters, storage precisions and the per-site arithmetic of one time step
// (forces of Eq. (FFF), shifted equilibrium and BGK collision of Eq. (be)).
// Both kernel families (generic and tiled) call the site functions below, so
// they compute bit-identical results for the same inputs.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace lbhb {

// ---------------------------------------------------------------- tables --
// D2Q9 order: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
__host__ __device__ constexpr int q_cx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int q_cy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int q_opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
__host__ __device__ constexpr double q_w(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// Half of the 24-neighbour interaction stencil (one vector of each +-c pair),
// k = 0..11; the first four (k < 4) have |c|^2 <= 2 and form belt 1.
__host__ __device__ constexpr int hs_dx(int k)
{
    return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 1 : k == 3 ? -1 : k == 4 ? 2 : k == 5 ? 0 : k == 6 ? 2 : k == 7 ? -2 : k == 8 ? 1 : k == 9 ? -1 : k == 10 ? 2 : -2;
}
__host__ __device__ constexpr int hs_dy(int k)
{
    return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 1 : k == 3 ? 1 : k == 4 ? 0 : k == 5 ? 2 : k == 6 ? 1 : k == 7 ? 1 : k == 8 ? 2 : k == 9 ? 2 : k == 10 ? 2 : 2;
}
// Belt-1 weights: the standard D2Q9 weights 1/9 (|c|^2 = 1), 1/36 (|c|^2 = 2).
__host__ __device__ constexpr double hs_w1(int k)
{
    return k >= 4 ? 0.0 : (hs_dx(k) * hs_dx(k) + hs_dy(k) * hs_dy(k) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}
// Two-belt weights of the 25-velocity isotropic set, same second moment 1/3:
// |c|^2 = 1, 2, 4, 5, 8 -> 4/63, 4/135, 1/180, 2/945, 1/15120.
__host__ __device__ constexpr double hs_w2(int k)
{
    return (hs_dx(k) * hs_dx(k) + hs_dy(k) * hs_dy(k)) == 1 ? 4.0 / 63.0
         : (hs_dx(k) * hs_dx(k) + hs_dy(k) * hs_dy(k)) == 2 ? 4.0 / 135.0
         : (hs_dx(k) * hs_dx(k) + hs_dy(k) * hs_dy(k)) == 4 ? 1.0 / 180.0
         : (hs_dx(k) * hs_dx(k) + hs_dy(k) * hs_dy(k)) == 5 ? 2.0 / 945.0
                                                            : 1.0 / 15120.0;
}

// ------------------------------------------------------------ parameters --
// Per-cell parameters as stored on the device, in both compute precisions so
// that FP32 kernels never touch the (slow) FP64 pipe for them.
template <class C> struct ParamSet {
    C tau, omega, rho0, inv_rho0, gab_over_rho0;  // tau, omega of species A
    C tau_b, omega_b;  // species B (equal to tau, omega unless a time per species is set)
    // weight of the other species' moments in the common velocity, seen from A and
    // from B: mix[0] = tau_A / tau_B, mix[1] = tau_B / tau_A (both 1 for one time)
    C mix[2];
    C g1[2], g2[2];  // G^a_ss, G^r_ss for s = A, B
    C u_wall;        // top wall +u_wall, bottom wall -u_wall (Couette)
    C rho_bar[2];    // FP16 shift reference
    C f0;            // Kolmogorov body force F_x(y) = f0 sin(pi y two_over_ny)
    C two_over_ny;
    // multiple-relaxation-time collision: per species s, (w - s_e)/12,
    // (w - s_eps)/12, (w - s_q)/12, (w - s_nu)/4 with w = omega_s (mrt_delta);
    // mrt != 0 if the cell sets any of the four rates
    C mrt_h[2][4];
    int mrt;
};
struct CellDev {
    ParamSet<double> d;
    ParamSet<float> f;
};
template <class C> __host__ __device__ inline const ParamSet<C>& params(const CellDev& c);
template <> __host__ __device__ inline const ParamSet<double>& params<double>(const CellDev& c) { return c.d; }
template <> __host__ __device__ inline const ParamSet<float>& params<float>(const CellDev& c) { return c.f; }

// Shift of the FP16 storage, g_i = f_i - w_i rho_bar_s, in the compute type;
// the same expression everywhere a population is stored or loaded.
template <class C> __device__ inline C pop_shift(int i, const ParamSet<C>& p, int s) { return C(q_w(i)) * p.rho_bar[s]; }

// Population array geometry: [cell][s][i][y][pitch], x fastest.
struct Geom {
    int nx, ny, pitch, n_cells;
    long long plane;       // ny * pitch
    long long cellstride;  // 18 * plane
};

__host__ __device__ inline long long fidx(const Geom& g, int cell, int q, int y, int x)
{
    return (long long)cell * g.cellstride + (long long)q * g.plane + (long long)y * g.pitch + x;
}

// ------------------------------------------------------- storage formats --
// Random bits for stochastic rounding.  A thread seeds one stream per row it
// stores from a hash of the site and of the site's current densities (so the
// stream changes from one step to the next without a step counter, and a run
// is reproducible bit for bit), then advances it by one 32-bit linear
// congruential step per stored value (the Numerical Recipes constants) and uses
// its top 13 bits.  The seed hash is the "lowbias32" integer finaliser found by
// C. Wellons' hash-prospector search.
struct Dither {
    uint32_t s;
    __device__ static uint32_t mix(uint32_t x)
    {
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        return x;
    }
    __device__ void seed(uint32_t site, uint32_t data) { s = mix(site ^ mix(data)); }
    __device__ uint32_t next13()
    {
        s = s * 1664525u + 1013904223u;
        return s >> 19;
    }
};

// FP32 -> FP16 with stochastic rounding: FP16 keeps the top 10 of the 23
// mantissa bits of a normal FP32 value; adding 13 uniform random bits below
// them and truncating rounds up with probability (dropped bits) / 2^13, so the
// stored value is the input in expectation.  Exact for inputs whose FP16 image
// is a normal number; below 2^-14 the dropped part is wider than the random
// bits and the rounding leans towards zero (callers scale values away from
// that range).
__device__ inline __half half_sr_round(float v, Dither& d)
{
    return __float2half_rz(__uint_as_float(__float_as_uint(v) + d.next13()));
}

// FP16 element of the stochastically rounded storage (a distinct type so that
// every kernel is instantiated for it).
struct half_sr {
    __half h;
};

template <class T> struct Store;
// scale: stored value = scale * (f - shift); dithered: stores round stochastically
template <> struct Store<float> {
    using C = float;
    static constexpr bool shifted = false, dithered = false;
    static constexpr float scale = 1.f;
    __device__ static C ld(const float* p, long long k, C) { return p[k]; }
    __device__ static void st(float* p, long long k, C v, C) { p[k] = v; }
    __device__ static void st(float* p, long long k, C v, C, Dither&) { p[k] = v; }
};
template <> struct Store<double> {
    using C = double;
    static constexpr bool shifted = false, dithered = false;
    static constexpr double scale = 1.0;
    __device__ static C ld(const double* p, long long k, C) { return p[k]; }
    __device__ static void st(double* p, long long k, C v, C) { p[k] = v; }
    __device__ static void st(double* p, long long k, C v, C, Dither&) { p[k] = v; }
};
// FP16 storage of the shifted populations g_i = f_i - w_i rho_bar_s.
template <> struct Store<__half> {
    using C = float;
    static constexpr bool shifted = true, dithered = false;
    static constexpr float scale = 1.f;
    __device__ static C ld(const __half* p, long long k, C shift) { return __half2float(p[k]) + shift; }
    __device__ static void st(__half* p, long long k, C v, C shift) { p[k] = __float2half_rn(v - shift); }
    __device__ static void st(__half* p, long long k, C v, C shift, Dither&) { p[k] = __float2half_rn(v - shift); }
};
// FP16 storage of 4096 g_i, rounded stochastically by the step kernels (round to
// nearest where a state is set from outside: initialisation and import).  The
// power-of-two scale is exact and moves every |g| >= 2^-26 into the FP16
// normal range, where the stochastic rounding is exact; |g| <= 16 fits.
template <> struct Store<half_sr> {
    using C = float;
    static constexpr bool shifted = true, dithered = true;
    static constexpr float scale = 4096.f;
    __device__ static C ld(const half_sr* p, long long k, C shift)
    {
        return __half2float(p[k].h) * (1.f / 4096.f) + shift;
    }
    __device__ static void st(half_sr* p, long long k, C v, C shift) { p[k].h = __float2half_rn((v - shift) * scale); }
    __device__ static void st(half_sr* p, long long k, C v, C shift, Dither& d)
    {
        p[k].h = half_sr_round((v - shift) * scale, d);
    }
};

// Stored element -> compute type (shift and scale not included).
__device__ inline float to_c(float v) { return v; }
__device__ inline double to_c(double v) { return v; }
__device__ inline float to_c(__half v) { return __half2float(v); }
__device__ inline float to_c(half_sr v) { return __half2float(v.h); }

// sin(pi x): the Kolmogorov profile sin(2 pi y / ny) is sin_pi(y * 2/ny).
template <class C> __device__ inline C sin_pi(C x);
template <> __device__ inline float sin_pi<float>(float x) { return sinpif(x); }
template <> __device__ inline double sin_pi<double>(double x) { return sinpi(x); }

// Body force density F_x of row y (zero when f0 = 0).
template <class C> __device__ inline C body_force_x(const ParamSet<C>& p, int y)
{
    return p.f0 == C(0) ? C(0) : p.f0 * sin_pi<C>(C(y) * p.two_over_ny);
}

template <class C> __device__ inline C expm1_c(C x);
template <> __device__ inline float expm1_c<float>(float x) { return expm1f(x); }
template <> __device__ inline double expm1_c<double>(double x) { return expm1(x); }

// 1 - e^{-t} in FP32 without the library's expm1f, for psi: Cody-Waite
// argument reduction t = k ln2 + r, |r| <= ln2/2 (k the nearest integer to
// t log2(e), rounded by adding 1.5 * 2^23; ln2 split so that k * OMX_LN2_HI is
// exact for |k| < 2^11), the Taylor polynomial of 1 - e^{-r} to degree 7
// (truncation below 2^-27 of the result for |r| <= ln2/2), and
//   1 - e^{-t} = (1 - 2^-k) + 2^-k (1 - e^{-r}),
// with 2^-k built in the exponent field from the integer bits of k that the
// rounding constant leaves in the low mantissa.  t is clamped to 80, beyond
// which 1 - e^{-t} rounds to 1.  Every operation is rounded to nearest once
// (explicit fma/mul/add), so the packed pair and the scalar forms agree bit
// for bit.  In an FP32 emulation of these steps the error stays within 1.2 ulp
// of the exact value for t in [1e-6, 40].
constexpr float OMX_LOG2E = 1.44269504088896340736f, OMX_ROUND = 12582912.0f;
constexpr float OMX_LN2_HI = 0.693145751953125f, OMX_LN2_LO = 1.42860682030941723212e-6f;
// Taylor coefficients of 1 - e^{-r}: (-1)^(n+1) / n!, n = 1..7
__host__ __device__ constexpr float omx_d(int n)
{
    return n == 1 ? 1.0f : n == 2 ? -0.5f : n == 3 ? 1.0f / 6.0f : n == 4 ? -1.0f / 24.0f : n == 5 ? 1.0f / 120.0f
         : n == 6 ? -1.0f / 720.0f : 1.0f / 5040.0f;
}

__device__ __forceinline__ float omx_pow2_neg(float km)
{
    return __uint_as_float(0x3f800000u - (__float_as_uint(km) << 23));
}
__device__ __forceinline__ float one_minus_exp_neg(float t)
{
    t = fminf(t, 80.f);
    const float km = __fmaf_rn(t, OMX_LOG2E, OMX_ROUND);
    const float k = __fsub_rn(km, OMX_ROUND);
    float r = __fmaf_rn(k, -OMX_LN2_HI, t);
    r = __fmaf_rn(k, -OMX_LN2_LO, r);
    float q = omx_d(7);
#pragma unroll
    for (int n = 6; n >= 1; --n) q = __fmaf_rn(q, r, omx_d(n));
    q = __fmul_rn(q, r);
    const float s = omx_pow2_neg(km);
    return __fmaf_rn(s, q, __fsub_rn(1.0f, s));
}

// psi(rho) = rho0 (1 - exp(-rho/rho0)): FP32 through one_minus_exp_neg, FP64
// as -rho0 expm1(-rho/rho0)
__device__ inline float psi_of(float rho, float rho0, float inv_rho0)
{
    return __fmul_rn(rho0, one_minus_exp_neg(__fmul_rn(rho, inv_rho0)));
}
__device__ inline double psi_of(double rho, double rho0, double inv_rho0) { return -rho0 * expm1(-rho * inv_rho0); }

// ------------------------------------------------------------ lane pairs --
// The tiled kernel's threads update one species at two adjacent sites (x, x+1)
// with identical arithmetic; P2<C> holds the pair.  For FP32 a pair is one
// 64-bit operand of the packed FP32 instructions of sm_100 and later
// (add/sub/mul/fma.rn.f32x2): one issued instruction yields both results, each
// rounded as the scalar instruction would round it.  FP64 pairs are two scalar
// operations.  The site arithmetic below is written once for a lane type V (a
// scalar for the one-site-per-thread kernel, P2 for the tiled kernel), with the
// multiply-adds explicit (vfma).
template <class C> struct P2;

template <> struct P2<float> {
    float2 v;
    P2() = default;
    __device__ explicit P2(double s) : v(make_float2((float)s, (float)s)) {}
    __device__ explicit P2(float s) : v(make_float2(s, s)) {}
    __device__ P2(float a, float b) : v(make_float2(a, b)) {}
    __device__ explicit P2(float2 w) : v(w) {}
    __device__ float a() const { return v.x; }
    __device__ float b() const { return v.y; }
};

template <> struct P2<double> {
    double x, y;
    P2() = default;
    __device__ explicit P2(double s) : x(s), y(s) {}
    __device__ P2(double a, double b) : x(a), y(b) {}
    __device__ double a() const { return x; }
    __device__ double b() const { return y; }
};

namespace pk {
__device__ __forceinline__ unsigned long long bits(float2 a)
{
    unsigned long long u;
    memcpy(&u, &a, 8);
    return u;
}
__device__ __forceinline__ float2 unbits(unsigned long long u)
{
    float2 a;
    memcpy(&a, &u, 8);
    return a;
}
}  // namespace pk

__device__ __forceinline__ P2<float> operator+(P2<float> a, P2<float> b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk::bits(a.v)), "l"(pk::bits(b.v)));
    return P2<float>(pk::unbits(d));
}
__device__ __forceinline__ P2<float> operator-(P2<float> a, P2<float> b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk::bits(a.v)), "l"(pk::bits(b.v)));
    return P2<float>(pk::unbits(d));
}
__device__ __forceinline__ P2<float> operator*(P2<float> a, P2<float> b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk::bits(a.v)), "l"(pk::bits(b.v)));
    return P2<float>(pk::unbits(d));
}
__device__ __forceinline__ P2<float> vfma(P2<float> a, P2<float> b, P2<float> c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk::bits(a.v)), "l"(pk::bits(b.v)), "l"(pk::bits(c.v)));
    return P2<float>(pk::unbits(d));
}
__device__ __forceinline__ P2<double> operator+(P2<double> a, P2<double> b) { return P2<double>(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ P2<double> operator-(P2<double> a, P2<double> b) { return P2<double>(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ P2<double> operator*(P2<double> a, P2<double> b) { return P2<double>(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ P2<double> vfma(P2<double> a, P2<double> b, P2<double> c)
{
    return P2<double>(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
// scalar type of a lane value
template <class V> struct LaneScalar { using type = V; };
template <class C> struct LaneScalar<P2<C>> { using type = C; };

__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Lane-wise helpers: reciprocal for the velocity (FP32 through the fast
// division intrinsic, 2 ulp; FP64 correctly rounded), psi_s/rho_s with its limit
// 1 at rho_s -> 0, and psi of the densities.
__device__ __forceinline__ float lane_rcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double lane_rcp(double x) { return 1.0 / x; }
template <class C> __device__ __forceinline__ P2<C> lane_rcp(P2<C> x) { return P2<C>(lane_rcp(x.a()), lane_rcp(x.b())); }

__device__ __forceinline__ float lane_por(float psi, float rho) { return rho != 0.f ? __fdividef(psi, rho) : 1.f; }
__device__ __forceinline__ double lane_por(double psi, double rho) { return rho != 0.0 ? psi / rho : 1.0; }
template <class C> __device__ __forceinline__ P2<C> lane_por(P2<C> psi, P2<C> rho)
{
    return P2<C>(lane_por(psi.a(), rho.a()), lane_por(psi.b(), rho.b()));
}

// psi of a pair of densities, each lane equal to psi_of: FP32 with every step
// of one_minus_exp_neg packed; FP64 through expm1 per lane
__device__ __forceinline__ P2<float> lane_psi(P2<float> rho, P2<float> rho0, P2<float> inv_rho0)
{
    P2<float> t = rho * inv_rho0;
    t = P2<float>(fminf(t.a(), 80.f), fminf(t.b(), 80.f));
    const P2<float> km = vfma(t, P2<float>(OMX_LOG2E), P2<float>(OMX_ROUND));
    const P2<float> k = km - P2<float>(OMX_ROUND);
    P2<float> r = vfma(k, P2<float>(-OMX_LN2_HI), t);
    r = vfma(k, P2<float>(-OMX_LN2_LO), r);
    P2<float> q = P2<float>(omx_d(7));
#pragma unroll
    for (int n = 6; n >= 1; --n) q = vfma(q, r, P2<float>(omx_d(n)));
    q = q * r;
    const P2<float> sk(omx_pow2_neg(km.a()), omx_pow2_neg(km.b()));
    return rho0 * vfma(sk, q, P2<float>(1.0f) - sk);
}
__device__ __forceinline__ P2<double> lane_psi(P2<double> rho, P2<double> rho0, P2<double> inv_rho0)
{
    return P2<double>(psi_of(rho.a(), rho0.a(), inv_rho0.a()), psi_of(rho.b(), rho0.b(), inv_rho0.b()));
}

// Pairs of adjacent elements to and from shared or global memory, in the
// compute type (FP16 storage converts both halves at once).
template <class T> struct Pair;
template <> struct Pair<float> {
    __device__ static P2<float> ld(const float* p) { return P2<float>(*reinterpret_cast<const float2*>(p)); }
    __device__ static void st(float* p, P2<float> v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <> struct Pair<double> {
    __device__ static P2<double> ld(const double* p)
    {
        const double2 v = *reinterpret_cast<const double2*>(p);
        return P2<double>(v.x, v.y);
    }
    __device__ static void st(double* p, P2<double> v) { *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y); }
};
template <> struct Pair<__half> {
    __device__ static P2<float> ld(const __half* p) { return P2<float>(__half22float2(*reinterpret_cast<const __half2*>(p))); }
};
template <> struct Pair<half_sr> {
    __device__ static P2<float> ld(const half_sr* p)
    {
        return P2<float>(__half22float2(*reinterpret_cast<const __half2*>(p)));
    }
};

// ----------------------------------------------------- per-site physics --
// Interaction sums of Eq. (FFF) at one site for one species, from the
// differences d_k = g(r + c_k) - g(r - c_k) over the half stencil:
//   S1 = sum_{belt 1} w c psi_s(r+c),  S2 = sum_{belts 1+2} p c psi_s(r+c),
//   X  = sum_{belt 1} w c rho_s'(r+c).
template <class V> struct Sums {
    V s1x, s1y, s2x, s2y, xx, xy;
};

template <class V>
__device__ inline Sums<V> stencil_sums(const V d[12], const V e[4])
{
    // Terms grouped by weight (the half stencil is symmetric under x -> -x):
    //   belt 1: (1,0),(0,1) weight 1/9; (1,1),(-1,1) weight 1/36
    //   belts 1+2: |c|^2 = 1: 4/63, 2: 4/135, 4: 1/180, 5: 2/945, 8: 1/15120
    const V p1 = V(hs_w2(0)), p2 = V(hs_w2(2)), p4x2 = V(2.0 * hs_w2(4)), p5 = V(hs_w2(6)), p8x2 = V(2.0 * hs_w2(10));
    const V w1 = V(hs_w1(0)), w2 = V(hs_w1(2)), two = V(2.0);
    const V dm23 = d[2] - d[3], dp23 = d[2] + d[3];          // (1,1), (-1,1)
    const V dm67 = d[6] - d[7], dp67 = d[6] + d[7];          // (2,1), (-2,1)
    const V dm89 = d[8] - d[9], dp89 = d[8] + d[9];          // (1,2), (-1,2)
    const V dm1011 = d[10] - d[11], dp1011 = d[10] + d[11];  // (2,2), (-2,2)
    Sums<V> r;
    r.s1x = vfma(w2, dm23, w1 * d[0]);
    r.s1y = vfma(w2, dp23, w1 * d[1]);
    r.s2x = vfma(p8x2, dm1011, vfma(p5, vfma(two, dm67, dm89), vfma(p4x2, d[4], vfma(p2, dm23, p1 * d[0]))));
    r.s2y = vfma(p8x2, dp1011, vfma(p5, vfma(two, dp89, dp67), vfma(p4x2, d[5], vfma(p2, dp23, p1 * d[1]))));
    r.xx = vfma(w2, e[2] - e[3], w1 * e[0]);
    r.xy = vfma(w2, e[2] + e[3], w1 * e[1]);
    return r;
}

// Multiple-relaxation-time correction of a BGK collision (the orthogonal D2Q9
// moments rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy of Lallemand and Luo,
// Phys. Rev. E 61 (2000) 6546; not in the paper).  The BGK result f + w d,
// d_i = f^eq_i - f_i, relaxes every moment with w; adding
//   -sum_k (s_k - w) n_k M_ki / D_k,   n_k = sum_i M_ki (f_i - f^eq_i),
// over k = e, eps, q_x, q_y, p_xx, p_xy (norms D = 36, 36, 12, 12, 4, 4) gives
// those moments their own rates s_k; rho and j keep w.  d_0 enters as
// -(d_1 + ... + d_8) (f and f^eq carry the same density).  h = ((w - s_e)/12,
// (w - s_eps)/12, (w - s_q)/12, (w - s_nu)/4).  fs[0] is left to the caller's
// closure (the correction has no density).
template <class V>
__device__ inline void mrt_delta(const V d[9], const V h[4], V fs[9])
{
    const V s13 = d[1] + d[3], s24 = d[2] + d[4], s57 = d[5] + d[7], s68 = d[6] + d[8];
    const V ax = s13 + s24, dg = s57 + s68;  // axis and diagonal sums
    const V d13 = d[1] - d[3], d24 = d[2] - d[4], d57 = d[5] - d[7], d86 = d[8] - d[6];
    const V ce = h[0] * vfma(V(2.0), dg, ax);               // e:   n = 3 (A + 2 Dg)
    const V cp = V(0.0) - h[1] * vfma(V(2.0), ax, dg);      // eps: n = -3 (2 A + Dg)
    const V cqx = h[2] * vfma(V(-2.0), d13, d57 + d86);     // q_x: -2 d13 + d57 + d86
    const V cqy = h[2] * vfma(V(-2.0), d24, d57 - d86);     // q_y: -2 d24 + d57 - d86
    const V cxx = h[3] * (s13 - s24), cxy = h[3] * (s57 - s68);  // p_xx, p_xy
    const V P = vfma(V(2.0), cp, ce), Q = V(0.0) - vfma(V(2.0), ce, cp);
    const V P1 = P - cxx, P2 = P + cxx, Q1 = Q - cxy, Q2 = Q + cxy;
    const V qs = cqx + cqy, qd = cqx - cqy;
    fs[1] = fs[1] + vfma(V(2.0), cqx, P1);
    fs[3] = fs[3] + vfma(V(-2.0), cqx, P1);
    fs[2] = fs[2] + vfma(V(2.0), cqy, P2);
    fs[4] = fs[4] + vfma(V(-2.0), cqy, P2);
    fs[5] = fs[5] + (Q1 - qs);
    fs[7] = fs[7] + (Q1 + qs);
    fs[6] = fs[6] + (Q2 + qd);
    fs[8] = fs[8] + (Q2 - qd);
}

// Shifted-velocity BGK collision of Eq. (be) for one species s at one site (or
// a pair of sites).
//   F_s    = -psi_s (G^a S1 + G^r S2) - (G_AB/rho0) rho_s X       (Eq. (FFF))
//   u_s    = u + tau F_s/rho_s = u + tau (a - (psi_s/rho_s)(G^a S1 + G^r S2) - (G_AB/rho0) X)
//   f*_is  = f_is + omega (f^eq_is(rho_s, u_s) - f_is),  omega = 1/tau, i = 1..8
// (tau, omega: the species' own relaxation time and rate; ntau = -tau)
//   f*_0s  = f_0s + sum_{i>=1} (f_is - f*_is)   (the BGK value in exact arithmetic)
// f^eq_i = w_i rho_s (1 + 3 c_i.u_s + 4.5 (c_i.u_s)^2 - 1.5 u_s^2) is evaluated for
// the pairs +-c_i together (even part + odd part).
// u is the common velocity of both species: j / (rho_A + rho_B) for one
// relaxation time (collide_site).
// ax = F_x / rho is the Kolmogorov body force per unit total density: species s
// receives rho_s ax of it (a share proportional to its density), which shifts
// its equilibrium velocity by tau ax.
// psi_s/rho_s is taken with its limit 1 at rho_s -> 0, so nothing divides by a
// vanishing species density.
// The rest population closes the mass.  FP32: each difference f_is - f*_is of
// nearby values is exact (Sterbenz), so the stored populations sum to the
// loaded ones up to the one rounding of f*_0s.  (Closing on the rounded sum
// rho_s instead repeats that sum's rounding at every site of a near-uniform
// state, which drifted the FP32 mass coherently by 4e-6 per 1000 steps.)  FP64,
// whose roundings are 2^29 times smaller and whose pipe bounds the step, closes
// on rho_s: f*_0s = rho_s - sum_{i>=1} f*_is (eight operations fewer).
// *Fx, *Fy receive F_s (for the force-corrected velocity of the observables).
// UNIT: tau = 1 (omega = 1, the paper's choice for all its runs), where the BGK
// update is f*_i = f^eq_i exactly and f_i only enters through the moments.
// MRT: the multiple-relaxation-time collision, the BGK one corrected by
// mrt_delta with the species' coefficients h[4] (before the rest population
// closes the mass).
template <class V, bool UNIT = false, bool MRT = false>
__device__ inline void collide_species(const V f[9], V rho_s, V psi_s, V ux, V uy, V ax, const Sums<V>& sm, V ga,
                                       V gr, V gx, V tau, V ntau, V omega, V fs[9], V* Fx, V* Fy,
                                       const V* h = nullptr)
{
    static_assert(!(UNIT && MRT), "the multiple-relaxation-time collision takes the general update");
    const V Gx = vfma(gr, sm.s2x, ga * sm.s1x);
    const V Gy = vfma(gr, sm.s2y, ga * sm.s1y);
    *Fx = rho_s * (ax - gx * sm.xx) - psi_s * Gx;
    *Fy = V(0.0) - vfma(psi_s, Gy, gx * rho_s * sm.xy);
    const V por = lane_por(psi_s, rho_s);
    const V hx = vfma(por, Gx, gx * sm.xx);
    const V hy = vfma(por, Gy, gx * sm.xy);
    const V usx = vfma(tau, ax - hx, ux);
    const V usy = vfma(ntau, hy, uy);
    // f^eq of a pair +-c: w rho (1 - 1.5 u^2 + 4.5 (c.u)^2) +- 3 w rho (c.u)
    const V base = vfma(V(-1.5), vfma(usx, usx, usy * usy), V(1.0));
    const V wr1 = V(q_w(1)) * rho_s, wr5 = V(q_w(5)) * rho_s;
    const V tr1 = V(3.0 * q_w(1)) * rho_s, tr5 = V(3.0 * q_w(5)) * rho_s;
    const V cu[4] = {usx, usy, usx + usy, usy - usx};  // c.u for i = 1, 2, 5, 6
    const int lo[4] = {1, 2, 5, 6}, hi[4] = {3, 4, 7, 8};
    constexpr bool exact_close = sizeof(typename LaneScalar<V>::type) == 4;
    V dsum = V(0.0), d[9];
    auto close = [&](int k) {
        const int i = lo[k], j = hi[k];
        if constexpr (exact_close) {
            const V dk = (f[i] - fs[i]) + (f[j] - fs[j]);
            dsum = k == 0 ? dk : dsum + dk;
        } else {
            dsum = k == 0 ? fs[i] + fs[j] : dsum + (fs[i] + fs[j]);
        }
    };
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const V a = (k < 2 ? wr1 : wr5) * vfma(V(4.5) * cu[k], cu[k], base);
        const V b = (k < 2 ? tr1 : tr5) * cu[k];
        const int i = lo[k], j = hi[k];
        if constexpr (UNIT) {
            fs[i] = a + b;
            fs[j] = a - b;
        } else {
            d[i] = (a + b) - f[i];
            d[j] = (a - b) - f[j];
            fs[i] = vfma(omega, d[i], f[i]);
            fs[j] = vfma(omega, d[j], f[j]);
        }
        if constexpr (!MRT) close(k);
    }
    if constexpr (MRT) {
        mrt_delta(d, h, fs);
#pragma unroll
        for (int k = 0; k < 4; ++k) close(k);
    }
    fs[0] = exact_close ? f[0] + dsum : rho_s - dsum;
}

// The same collision for shifted populations g_i = f_i - w_i rho_bar (FP16
// storage), computed on g directly: with dr = rho_s - rho_bar,
//   g^eq_i = f^eq_i - w_i rho_bar = w_i (dr + rho_s (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)),
//   g*_i = g_i + omega (g^eq_i - g_i),  g*_0 = g_0 + sum_{i>=1} (g_i - g*_i),
// so no population needs its shift added or removed, and the arithmetic works
// on the small deviations.  Momenta of g equal those of f (opposite directions
// carry equal weights).
// With scale != 1 the populations are scale * g (FP16 storage with stochastic
// rounding) and so are the results; rho_s, psi_s, u and the forces are not scaled.
// MRT as in collide_species (g - g^eq = f - f^eq, so the correction is the same).
template <class V, bool UNIT = false, bool MRT = false>
__device__ inline void collide_species_shifted(const V g[9], V rho_s, V rho_bar, V psi_s, V ux, V uy, V ax,
                                               const Sums<V>& sm, V ga, V gr, V gx, V tau, V ntau, V omega,
                                               V gs[9], V* Fx, V* Fy, V scale, const V* h = nullptr)
{
    static_assert(!(UNIT && MRT), "the multiple-relaxation-time collision takes the general update");
    const V Gx = vfma(gr, sm.s2x, ga * sm.s1x);
    const V Gy = vfma(gr, sm.s2y, ga * sm.s1y);
    *Fx = rho_s * (ax - gx * sm.xx) - psi_s * Gx;
    *Fy = V(0.0) - vfma(psi_s, Gy, gx * rho_s * sm.xy);
    const V por = lane_por(psi_s, rho_s);
    const V hx = vfma(por, Gx, gx * sm.xx);
    const V hy = vfma(por, Gy, gx * sm.xy);
    const V usx = vfma(tau, ax - hx, ux);
    const V usy = vfma(ntau, hy, uy);
    const V dr = (rho_s - rho_bar) * scale, rs = rho_s * scale;
    const V nusq = V(-1.5) * vfma(usx, usx, usy * usy);
    const V tr1 = V(3.0 * q_w(1)) * rs, tr5 = V(3.0 * q_w(5)) * rs;
    const V cu[4] = {usx, usy, usx + usy, usy - usx};  // c.u for i = 1, 2, 5, 6
    const int lo[4] = {1, 2, 5, 6}, hi[4] = {3, 4, 7, 8};
    V dsum = V(0.0), d[9];
    auto close = [&](int k) {
        const int i = lo[k], j = hi[k];
        const V dk = (g[i] - gs[i]) + (g[j] - gs[j]);
        dsum = k == 0 ? dk : dsum + dk;
    };
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const V a = V(k < 2 ? q_w(1) : q_w(5)) * vfma(rs, vfma(V(4.5) * cu[k], cu[k], nusq), dr);
        const V b = (k < 2 ? tr1 : tr5) * cu[k];
        const int i = lo[k], j = hi[k];
        if constexpr (UNIT) {
            gs[i] = a + b;
            gs[j] = a - b;
        } else {
            d[i] = (a + b) - g[i];
            d[j] = (a - b) - g[j];
            gs[i] = vfma(omega, d[i], g[i]);
            gs[j] = vfma(omega, d[j], g[j]);
        }
        if constexpr (!MRT) close(k);
    }
    if constexpr (MRT) {
        mrt_delta(d, h, gs);
#pragma unroll
        for (int k = 0; k < 4; ++k) close(k);
    }
    gs[0] = g[0] + dsum;
}

// Momentum of one species' populations, as differences of opposite directions
// (a state at rest gives exactly zero).
template <class V> __device__ inline V mom_x(const V f[9]) { return (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]); }
template <class V> __device__ inline V mom_y(const V f[9]) { return (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]); }

// Result of colliding one site: post-collision populations and the total
// force (for the force-corrected velocity of the observables).
template <class C> struct Collided {
    C fs[2][9];
    C Fx, Fy;
};

// Both species at one site: the common velocity u, then collide_species each.
// With one relaxation time u = j / (rho_A + rho_B).  With a time per species u
// is the Shan-Doolen common velocity (j_A/tau_A + j_B/tau_B) / (rho_A/tau_A +
// rho_B/tau_B), taken as (j_A + r j_B) / (rho_A + r rho_B), r = tau_A/tau_B
// (r = 1 gives the one-time velocity exactly), so that the collision conserves
// the total momentum; the Kolmogorov force is still shared as rho_s / rho.
// A cell with multiple-relaxation-time rates (p.mrt) takes the MRT collision.
template <class C>
__device__ inline void collide_site(const C f[2][9], const C rho[2], const C psi[2],
                                    const Sums<C> sm[2], const ParamSet<C>& p, C fx_body, Collided<C>& out)
{
    const C r = p.mix[0];
    const C jx = vfma(r, mom_x<C>(f[1]), mom_x<C>(f[0]));
    const C jy = vfma(r, mom_y<C>(f[1]), mom_y<C>(f[0]));
    const C inv_rw = lane_rcp(vfma(r, rho[1], rho[0]));
    const C ux = jx * inv_rw, uy = jy * inv_rw;
    const C ax = r == C(1) ? fx_body * inv_rw : fx_body * lane_rcp(rho[0] + rho[1]);
    C Fx[2], Fy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const C tau = s ? p.tau_b : p.tau, omega = s ? p.omega_b : p.omega;
        if (p.mrt)
            collide_species<C, false, true>(f[s], rho[s], psi[s], ux, uy, ax, sm[s], p.g1[s], p.g2[s],
                                            p.gab_over_rho0, tau, -tau, omega, out.fs[s], &Fx[s], &Fy[s],
                                            p.mrt_h[s]);
        else if (omega == C(1))
            collide_species<C, true>(f[s], rho[s], psi[s], ux, uy, ax, sm[s], p.g1[s], p.g2[s], p.gab_over_rho0,
                                     tau, -tau, omega, out.fs[s], &Fx[s], &Fy[s]);
        else
            collide_species<C, false>(f[s], rho[s], psi[s], ux, uy, ax, sm[s], p.g1[s], p.g2[s], p.gab_over_rho0,
                                      tau, -tau, omega, out.fs[s], &Fx[s], &Fy[s]);
    }
    out.Fx = Fx[0] + Fx[1];
    out.Fy = Fy[0] + Fy[1];
}

// Halfway bounce-back with a moving wall: a population f*_i leaving through the
// wall returns as f_opp(i) = f*_i - 2 w_i rho_s (c_i . u_w)/cs^2 (cs^2 = 1/3);
// *dpx receives the x-momentum this link delivers to the fluid.
template <class C>
__device__ inline C bounce(int i, C fstar, C rho_s, C u_w, C* dpx)
{
    const C back = fstar - C(6.0 * q_w(i)) * rho_s * (C(q_cx(i)) * u_w);
    *dpx = C(q_cx(q_opp(i))) * back - C(q_cx(i)) * fstar;
    return back;
}

// Row seen by the interaction stencil: periodic, or mirrored across the walls
// (psi(x,-k) = psi(x,k-1), psi(x,ny-1+k) = psi(x,ny-k)).  |y - in-range| <= 3.
__host__ __device__ inline int stencil_row(int y, int ny, int bc)
{
    if (bc == 0) return y < 0 ? y + ny : (y >= ny ? y - ny : y);
    return y < 0 ? -y - 1 : (y >= ny ? 2 * ny - y - 1 : y);
}
__host__ __device__ inline int wrap_x(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// Rows of a population buffer that a step updates, and where they sit in the
// global cell.  A whole cell: the buffer holds rows 0..ny-1, all updated
// (ylo = 0, nown = nyg = ny, y0g = 0, slab = 0).  A slab of one cell split into
// horizontal slabs: the buffer holds rows y0g-2 .. y0g+nown+1 of the global cell
// (two ghost rows on each side, ylo = 2); the step updates the nown rows in the
// middle, reads the ghost rows for the interaction stencil (they are copies of
// the neighbouring slabs' rows) and streams into them the populations that leave
// the slab, which the neighbours take over.
struct RowMap {
    int ylo, nown, y0g, nyg, slab;
};

// Buffer row the interaction stencil reads for buffer row e: a whole cell wraps
// periodically or mirrors at the walls; a slab reads its ghost rows, except
// beyond a Couette wall of the global cell, where the mirror rows are its own.
__host__ __device__ inline int stencil_load_row(int e, int ny, const RowMap& m, int bc)
{
    if (!m.slab) return stencil_row(e, ny, bc);
    const int gy = e - m.ylo + m.y0g;
    if (bc == 1 && (gy < 0 || gy >= m.nyg)) return stencil_row(gy, m.nyg, 1) - m.y0g + m.ylo;
    return e;
}

// Sum over the 32 lanes of a warp (result valid in lane 0).  FP32 values are
// added as an unevaluated (hi, lo) pair with the error-free two-sum, so the
// result carries ~2^-48 relative error without using the FP64 pipe; FP64
// values are added in FP64.
__device__ inline double warp_sum_compensated(float v)
{
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const float sum = __fadd_rn(hi, h2);
        const float bp = __fsub_rn(sum, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bp)), __fsub_rn(h2, bp));
        hi = sum;
        lo = __fadd_rn(__fadd_rn(lo, l2), err);
    }
    return (double)hi + (double)lo;
}
// Same for the sum of two values per lane (a + b is the first two-sum).
__device__ inline double warp_sum_compensated2(float a, float b)
{
    float hi = __fadd_rn(a, b);
    const float bp = __fsub_rn(hi, a);
    float lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bp)), __fsub_rn(b, bp));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const float sum = __fadd_rn(hi, h2);
        const float bq = __fsub_rn(sum, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bq)), __fsub_rn(h2, bq));
        hi = sum;
        lo = __fadd_rn(__fadd_rn(lo, l2), err);
    }
    return (double)hi + (double)lo;
}
__device__ inline double warp_sum_compensated2(double a, double b)
{
    double v = a + b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline double warp_sum_compensated(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Device error word bits.
enum : unsigned { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

}  // namespace lbhb
