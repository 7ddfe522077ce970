// Flow-curve surrogate kernels (include/lbhb_mlp.h): BF16 tensor-core products
// (mma.sync m16n8k16) with FP32 accumulation for the forward pass, serving,
// and a training step (forward, loss, backward) fused into one kernel per slab
// of the batch, followed by an ordered reduction with Adam on FP32 master
// weights.
//
// The layered forward pass (mlp_forward) writes every product as C[m][n] =
// sum_k A[m][k] B[n][k] with both operands K-contiguous ("NT"): activations
// [batch][in] times weights [out][in], with fused bias/tanh epilogues.  Batch
// rows beyond the live batch are written as zeros, so padded rows and columns
// never contribute.  Gradients are sums of per-CTA partials reduced in a fixed
// order, so results are reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbhb_mlp.h"
#include "lb_internal.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int NIN = 5, KIN = 16, HID = 128, NOUT = 2, NOUTP = 16;
constexpr long long OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * NIN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
                    OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID, OFF_W4 = OFF_B3 + HID,
                    OFF_B4 = OFF_W4 + NOUT * HID, NPARAM = OFF_B4 + NOUT;

struct LayerDef {
    int in, in_p, out, out_p;
    long long offW, offB;
};
__host__ __device__ constexpr LayerDef layer_def(int l)
{
    return l == 0   ? LayerDef{NIN, KIN, HID, HID, OFF_W1, OFF_B1}
           : l == 1 ? LayerDef{HID, HID, HID, HID, OFF_W2, OFF_B2}
           : l == 2 ? LayerDef{HID, HID, HID, HID, OFF_W3, OFF_B3}
                    : LayerDef{HID, HID, NOUT, NOUTP, OFF_W4, OFF_B4};
}

enum { EPI_TANH = 0, EPI_OUT = 1 };

struct Epi {
    const float* bias;  // EPI_TANH, EPI_OUT: [N]
    bf16* out_b;        // EPI_TANH: [rows][ld_out]
    bf16* out_t;        // EPI_TANH: [N][ld_t] (transposed copy)
    float* out_f;       // EPI_OUT: [rows][ld_out]
    int ld_out, ld_t;
    int rows_live;      // batch rows that hold data; later rows are written as zero
    int rows_buf;       // rows the buffers have
};

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// tanh on the special-function unit (tanh.approx.f32: relative error about
// 2^-11, a quarter of the BF16 rounding the activation then takes), for the
// training kernel's forward pass.  There its one instruction keeps the kernel's
// code short (a CTA runs the body once, so the code's length is fetch time);
// serving and the layered pass, whose bodies are short anyway, measured faster
// with tanhf and keep it.
__device__ __forceinline__ float act_tanh(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// C[m][n] = sum_{k in split} A[m][k] B[n][k]; 64x64 tile per CTA, 4 warps of
// 32x32, BK = 32.  K, the split chunk and both leading dimensions are multiples
// of 8 (16-byte vector loads).
template <int EPI>
__global__ void __launch_bounds__(128) gemm_nt(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
                                               int ldb, int M, int N, int K, int kchunk, Epi ep)
{
    __shared__ __align__(16) bf16 As[64][40];
    __shared__ __align__(16) bf16 Bs[64][40];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = kbeg; k0 < kend; k0 += 32) {
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int c = tid + rep * 128, r = c >> 2, kk = (c & 3) * 8;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < M && k0 + kk < kend) va = *reinterpret_cast<const uint4*>(A + (long long)(m0 + r) * lda + k0 + kk);
            if (n0 + r < N && k0 + kk < kend) vb = *reinterpret_cast<const uint4*>(B + (long long)(n0 + r) * ldb + k0 + kk);
            *reinterpret_cast<uint4*>(&As[r][kk]) = va;
            *reinterpret_cast<uint4*>(&Bs[r][kk]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < 32; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int rb = wm * 32 + mi * 16;
                a[mi][0] = *reinterpret_cast<const uint32_t*>(&As[rb + g][ks + 2 * t4]);
                a[mi][1] = *reinterpret_cast<const uint32_t*>(&As[rb + g + 8][ks + 2 * t4]);
                a[mi][2] = *reinterpret_cast<const uint32_t*>(&As[rb + g][ks + 2 * t4 + 8]);
                a[mi][3] = *reinterpret_cast<const uint32_t*>(&As[rb + g + 8][ks + 2 * t4 + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int cb = wn * 32 + ni * 8;
                b[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[cb + g][ks + 2 * t4]);
                b[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[cb + g][ks + 2 * t4 + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_bf16(acc[mi][ni], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b[ni][0], b[ni][1]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm * 32 + mi * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + ni * 8 + 2 * t4 + (r & 1);
                if (col >= N) continue;
                float v = acc[mi][ni][r];
                if (row >= ep.rows_buf) continue;
                const bool live = row < ep.rows_live;
                if (EPI == EPI_TANH)
                    v = live ? tanhf(v + ep.bias[col]) : 0.f;
                else
                    v = live ? v + ep.bias[col] : 0.f;
                if (EPI == EPI_OUT) {
                    ep.out_f[(long long)row * ep.ld_out + col] = v;
                } else {
                    const bf16 hv = __float2bfloat16_rn(v);
                    ep.out_b[(long long)row * ep.ld_out + col] = hv;
                    ep.out_t[(long long)col * ep.ld_t + row] = hv;
                }
            }
}

// z = (x - center) / half_range, padded to 16 columns, both layouts.
__global__ void normalise_kernel(const float* __restrict__ x, int B, int Bbuf, const float* __restrict__ center,
                                 const float* __restrict__ half, bf16* __restrict__ z, bf16* __restrict__ zt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bbuf) return;
    for (int c = 0; c < KIN; ++c) {
        float v = 0.f;
        if (b < B && c < NIN) v = (x[b * NIN + c] - center[c]) / half[c];
        const bf16 hv = __float2bfloat16_rn(v);
        z[(long long)b * KIN + c] = hv;
        zt[(long long)c * Bbuf + b] = hv;
    }
}

__device__ __forceinline__ float bce_logits(float z, float y)
{
    return fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
}

// FP32 masters -> padded BF16 weights [out_p][in_p], their transposes, padded FP32 biases.
__global__ void refresh_kernel(const float* __restrict__ p, bf16* w1, bf16* w1t, bf16* w2, bf16* w2t, bf16* w3,
                               bf16* w3t, bf16* w4, bf16* w4t, float* b1, float* b2, float* b3, float* b4)
{
    bf16* W[4] = {w1, w2, w3, w4};
    bf16* Wt[4] = {w1t, w2t, w3t, w4t};
    float* Bp[4] = {b1, b2, b3, b4};
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int base = 0;
    for (int l = 0; l < 4; ++l) {
        const LayerDef L = layer_def(l);
        const int nw = L.out_p * L.in_p;
        if (k >= base && k < base + nw) {
            const int o = (k - base) / L.in_p, i = (k - base) % L.in_p;
            const float v = (o < L.out && i < L.in) ? p[L.offW + (long long)o * L.in + i] : 0.f;
            const bf16 hv = __float2bfloat16_rn(v);
            W[l][o * L.in_p + i] = hv;
            Wt[l][i * L.out_p + o] = hv;
        }
        base += nw;
        if (k >= base && k < base + L.out_p) {
            const int o = k - base;
            Bp[l][o] = o < L.out ? p[L.offB + o] : 0.f;
        }
        base += L.out_p;
    }
}

__global__ void output_kernel(const float* __restrict__ out, int B, float scale, float* __restrict__ y)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    y[2 * b] = out[(long long)b * NOUTP] * scale;
    y[2 * b + 1] = out[(long long)b * NOUTP + 1];
}

constexpr int MAX_BINS = 256;  // bins of the serving error-budget table

}  // namespace

// ------------------------------------------------------------- serving --
// The whole serving call in one kernel: a CTA takes 64 queries through the
// normalisation, the three tanh layers and the output layer with every
// activation kept in shared memory (each warp owns 16 rows), the layer's
// weights staged in shared memory, then makes the fallback decision.  The
// products are the GEMM kernel's, tile for tile: one m16n8k16 BF16 product per
// 16-wide slice of K in increasing K, bias and tanh in FP32, activations
// rounded to BF16; so the served values equal the layered forward pass bit for
// bit.
constexpr int SRV_ROWS = 64, SRV_LD = HID + 8;  // padded rows: no bank conflicts on fragment loads
// two activation buffers and two weight buffers (the next layer's weights are
// copied while the current layer computes)
constexpr size_t SRV_SMEM = sizeof(bf16) * (2 * SRV_ROWS * SRV_LD + 2 * HID * SRV_LD);

// 16-byte asynchronous global -> shared copies, in commit groups
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Weights of layer l into a padded shared buffer, by all 128 threads.
__device__ __forceinline__ void stage_weights(bf16* Ws, const bf16* W, int l, int tid)
{
    const LayerDef L = layer_def(l);
    for (int e = tid; e < L.out_p * (L.in_p / 8); e += 128) {
        const int n = e / (L.in_p / 8), k8 = (e % (L.in_p / 8)) * 8;
        cp_async16(&Ws[n * SRV_LD + k8], W + (long long)n * L.in_p + k8);
    }
}

struct ServeArgs {
    const float* x;
    int B;
    const bf16* W[4];
    const float* bias[4];
    const float *center, *half;
    float scale, margin;
    const int* over_budget;
    int n_bins;
    float ls_lo, ls_hi;
    float *stress, *logit;
    int* fallback;
};

__global__ void __launch_bounds__(128) serve_fused_kernel(ServeArgs a)
{
    extern __shared__ __align__(16) unsigned char srv_smem[];
    bf16* act0 = reinterpret_cast<bf16*>(srv_smem);
    bf16* act1 = act0 + SRV_ROWS * SRV_LD;
    bf16* const wbuf0 = act1 + SRV_ROWS * SRV_LD;
    bf16* const wbuf1 = wbuf0 + HID * SRV_LD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int b0 = blockIdx.x * SRV_ROWS, r0 = warp * 16;
    // the first two layers' weights start copying at once
    stage_weights(wbuf0, a.W[0], 0, tid);
    cp_async_commit();
    stage_weights(wbuf1, a.W[1], 1, tid);
    cp_async_commit();

    // z = (x - center) / half_range, padded to KIN columns (zero rows past B)
    for (int e = tid; e < SRV_ROWS * KIN; e += 128) {
        const int r = e / KIN, c = e % KIN, b = b0 + r;
        float v = 0.f;
        if (b < a.B && c < NIN) v = (a.x[b * NIN + c] - a.center[c]) / a.half[c];
        act0[r * SRV_LD + c] = __float2bfloat16_rn(v);
    }
    bf16* in = act0;
    bf16* out = act1;
    for (int l = 0; l < 4; ++l) {
        const LayerDef L = layer_def(l);
        const bf16* Ws = (l & 1) ? wbuf1 : wbuf0;
        if (l < 3)
            cp_async_wait<1>();  // this layer's group is done, the next one may still fly
        else
            cp_async_wait<0>();
        __syncthreads();  // weights and input activations visible to all warps
        constexpr int NT = HID / 8;
        float acc[NT][4];
#pragma unroll
        for (int ni = 0; ni < NT; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[ni][r] = 0.f;
        const int nt = L.out_p / 8;
        for (int ks = 0; ks < L.in_p; ks += 16) {
            const uint32_t x0 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g) * SRV_LD + ks + 2 * t4]);
            const uint32_t x1 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g + 8) * SRV_LD + ks + 2 * t4]);
            const uint32_t x2 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g) * SRV_LD + ks + 2 * t4 + 8]);
            const uint32_t x3 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g + 8) * SRV_LD + ks + 2 * t4 + 8]);
#pragma unroll
            for (int ni = 0; ni < NT; ++ni) {
                if (ni >= nt) break;
                const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&Ws[(ni * 8 + g) * SRV_LD + ks + 2 * t4]);
                const uint32_t w1 = *reinterpret_cast<const uint32_t*>(&Ws[(ni * 8 + g) * SRV_LD + ks + 2 * t4 + 8]);
                mma_bf16(acc[ni], x0, x1, x2, x3, w0, w1);
            }
        }
        if (l < 3) {
#pragma unroll
            for (int ni = 0; ni < NT; ++ni)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int row = r0 + g + (r >= 2 ? 8 : 0), col = ni * 8 + 2 * t4 + (r & 1);
                    out[row * SRV_LD + col] = __float2bfloat16_rn(tanhf(acc[ni][r] + a.bias[l][col]));
                }
            __syncwarp();  // a warp reads back only its own rows
            bf16* t = in;
            in = out;
            out = t;
            if (l + 2 < 4) {
                __syncthreads();  // every warp is done with this layer's weights
                stage_weights((l & 1) ? wbuf1 : wbuf0, a.W[l + 2], l + 2, tid);
                cp_async_commit();
            }
        } else {
            // columns 0 (stress / scale) and 1 (logit) sit in n-tile 0: lanes with t4 == 0
            if (t4 == 0) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int row = r0 + g + 8 * h2, b = b0 + row;
                    if (b >= a.B) continue;
                    const float y0 = acc[0][2 * h2] + a.bias[3][0], y1 = acc[0][2 * h2 + 1] + a.bias[3][1];
                    bool outside = false;
                    for (int c = 0; c < NIN; ++c) {
                        const float xv = a.x[b * NIN + c];
                        outside |= !(fabsf(xv - a.center[c]) <= a.half[c]);
                    }
                    bool budget = false;
                    if (a.n_bins > 0) {
                        const float ls = a.x[b * NIN];
                        int k = (int)floorf((ls - a.ls_lo) / (a.ls_hi - a.ls_lo) * a.n_bins);
                        k = k < 0 ? 0 : (k >= a.n_bins ? a.n_bins - 1 : k);
                        budget = a.over_budget[k] != 0;
                    }
                    a.stress[b] = y0 * a.scale;
                    a.logit[b] = y1;
                    a.fallback[b] = (outside || budget || !(fabsf(y1) >= a.margin)) ? 1 : 0;
                }
            }
        }
    }
}

// ------------------------------------------------------------ training --
// Loss gradient and backpropagation in one kernel: a CTA takes a slab of 64
// batch rows (each warp 16) through the normalisation, the forward pass, the
// loss and the backward pass with every activation in shared memory, and adds
// the slab's contribution to every weight and bias gradient into its own row
// of FP32 partial sums; grad_finish_kernel then sums the rows in a fixed order
// (reproducible) and, for a training step, applies Adam and refreshes the BF16
// weight copies.  The products are the layered kernels': BF16 operands, FP32
// accumulation, activations and pre-activation gradients rounded to BF16.
//   forward   H_l = tanh(X_l W_l^T + b_l) (rows past the batch are zero)
//   loss      (y0 - t)^2 + lam BCE(y1, label), mean over the batch
//   backward  dW_l = D_l^T X_l, db_l = column sums of D_l,
//             D_{l-1} = (D_l W_l) * (1 - H_{l-1}^2)
// The weight gradients multiply two row-major slab buffers along the batch
// (the contraction index is their row), so both operands are loaded with
// ldmatrix.trans.  Each pre-activation gradient overwrites, row by row, the
// activation it was computed from once every warp has used that activation.
constexpr int TR_ROWS = 64;          // batch rows per slab
constexpr int TR_LD = HID + 8;       // padded 128-wide rows (activations, weights)
constexpr int TR_LDZ = KIN + 8;      // padded 16-wide rows (inputs, output gradient)
constexpr int TR_MAX_CTAS = 304;     // persistent CTAs at most (two per SM), one partial row each
// inputs, output gradient, three activations and one weight buffer: 90 KB, two CTAs per SM
constexpr size_t TR_SMEM = sizeof(bf16) * (2 * TR_ROWS * TR_LDZ + 3 * TR_ROWS * TR_LD + HID * TR_LD);

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const bf16* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t r[4], const bf16* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}

// A rows x cols BF16 matrix (cols a multiple of 8) into a padded shared buffer.
__device__ __forceinline__ void stage_matrix(bf16* Ws, const bf16* W, int rows, int cols, int tid)
{
    for (int e = tid; e < rows * (cols / 8); e += 128) {
        const int r = e / (cols / 8), c8 = (e % (cols / 8)) * 8;
        cp_async16(&Ws[r * TR_LD + c8], W + (long long)r * cols + c8);
    }
}

struct TrainArgs {
    const float *x, *target, *label;
    int B;
    const bf16* W[4];   // [out_p][in_p]
    const bf16* Wt[4];  // [in_p][out_p]
    const float* bias[4];
    const float *center, *half;
    float inv_scale, lam;
    float* part;        // [gridDim.x][NPARAM] partial gradients
    double* loss_part;  // [gridDim.x]
};

// One warp's 16 x N product of its rows of `in` (K wide) with the staged weights
// Ws [N][K]: acc[n-tile][4], K-steps of 16 in increasing order (NT even).  The
// operand fragments come from ldmatrix: the A tile as four 8 x 8 matrices (rows
// 0-7 | 8-15) x (k 0-7 | 8-15), two n-tiles of B per load.
template <int NT>
__device__ __forceinline__ void rows_times_weights(float (&acc)[NT][4], const bf16* in, int ld_in, int K,
                                                   const bf16* Ws, int r0, int lane)
{
#pragma unroll
    for (int ni = 0; ni < NT; ++ni)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[ni][r] = 0.f;
    const int j = lane >> 3, rr = lane & 7;
    for (int ks = 0; ks < K; ks += 16) {
        uint32_t a[4];
        ldsm_x4(a, in + (r0 + rr + (j & 1) * 8) * ld_in + ks + (j >> 1) * 8);
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
            uint32_t b[4];  // (n 0-7, k 0-7 | 8-15), (n 8-15, k 0-7 | 8-15) of the n-tile pair
            ldsm_x4(b, Ws + (np * 16 + rr + (j >> 1) * 8) * TR_LD + ks + (j & 1) * 8);
            mma_bf16(acc[2 * np], a[0], a[1], a[2], a[3], b[0], b[1]);
            mma_bf16(acc[2 * np + 1], a[0], a[1], a[2], a[3], b[2], b[3]);
        }
    }
}

// A weight-gradient block dW[m0 + 16 MT][n0 + 8 NT] = sum over the slab's 64
// rows b of D[b][o] X[b][i]: A = D^T and B = X loaded with ldmatrix.trans from
// the row-major slab buffers (NT even).
template <int MT, int NT>
__device__ __forceinline__ void slab_outer(float (&acc)[MT][NT][4], const bf16* D, int ldD, int m0, const bf16* X,
                                           int ldX, int n0, int lane)
{
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int ni = 0; ni < NT; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mi][ni][r] = 0.f;
    const int j = lane >> 3, rr = lane & 7;
#pragma unroll
    for (int k0 = 0; k0 < TR_ROWS; k0 += 16) {
        uint32_t a[MT][4];
#pragma unroll
        for (int mi = 0; mi < MT; ++mi)  // matrices (m 0-7|8-15) x (k 0-7|8-15): a0..a3
            ldsm_x4_trans(a[mi], D + (k0 + rr + ((j >> 1) & 1) * 8) * ldD + m0 + mi * 16 + (j & 1) * 8);
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {  // two n-tiles: (k 0-7|8-15) x (n 0-7|8-15)
            uint32_t b[4];
            ldsm_x4_trans(b, X + (k0 + rr + (j & 1) * 8) * ldX + n0 + np * 16 + (j >> 1) * 8);
#pragma unroll
            for (int mi = 0; mi < MT; ++mi) {
                mma_bf16(acc[mi][2 * np], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b[0], b[1]);
                mma_bf16(acc[mi][2 * np + 1], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b[2], b[3]);
            }
        }
    }
}

// Adds (first slab: stores) a weight-gradient block to the CTA's partial row;
// entries outside the live out x in block are skipped.
template <int MT, int NT, int LS>
__device__ __forceinline__ void put_wgrad(float* row, const float (&acc)[MT][NT][4], long long offW, int m0, int n0,
                                          int g, int t4, bool first)
{
    constexpr LayerDef L = layer_def(LS);  // the block's shape; offW places it
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int ni = 0; ni < NT; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // rows g and g + 8: the pair (i, i + 1) of adjacent columns
                const int o = m0 + mi * 16 + g + 8 * h, i = n0 + ni * 8 + 2 * t4;
                if (o >= L.out || i >= L.in) continue;
                float* p = row + offW + (long long)o * L.in + i;
                const float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (i + 1 < L.in && ((offW + (long long)o * L.in + i) & 1) == 0) {  // one 8-byte access
                    float2* p2 = reinterpret_cast<float2*>(p);
                    if (first) {
                        *p2 = make_float2(v0, v1);
                    } else {
                        const float2 q = *p2;
                        *p2 = make_float2(q.x + v0, q.y + v1);
                    }
                } else {
                    p[0] = first ? v0 : p[0] + v0;
                    if (i + 1 < L.in) p[1] = first ? v1 : p[1] + v1;
                }
            }
}

// Bias gradient of layer l: column sums of the slab's D (rows in increasing order).
__device__ __forceinline__ void put_bgrad(float* row, const bf16* D, int ld, int l, int tid, bool first)
{
    const LayerDef L = layer_def(l);
    if (tid >= L.out) return;
    float s = 0.f;
    for (int b = 0; b < TR_ROWS; ++b) s += __bfloat162float(D[b * ld + tid]);
    float* p = row + L.offB + tid;
    *p = first ? s : *p + s;
}

// D_{l-1} = (D_l W_l) * (1 - H^2) for the warp's rows, written over H (BF16).
template <int NT>
__device__ __forceinline__ void back_rows(const bf16* D, int ldD, int K, const bf16* Wts, bf16* H, int r0, int g,
                                          int t4, int b0, int B)
{
    float acc[NT][4];
    rows_times_weights<NT>(acc, D, ldD, K, Wts, r0, (g << 2) | t4);
#pragma unroll
    for (int ni = 0; ni < NT; ++ni)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = r0 + g + (r >= 2 ? 8 : 0), col = ni * 8 + 2 * t4 + (r & 1);
            const float h = __bfloat162float(H[row * TR_LD + col]);
            const float v = b0 + row < B ? acc[ni][r] * (1.f - h * h) : 0.f;
            H[row * TR_LD + col] = __float2bfloat16_rn(v);
        }
}

__global__ void __launch_bounds__(128, 2) train_fused_kernel(TrainArgs a)
{
    extern __shared__ __align__(16) unsigned char tr_smem[];
    bf16* const Zs = reinterpret_cast<bf16*>(tr_smem);        // [64][TR_LDZ] inputs
    bf16* const D4 = Zs + TR_ROWS * TR_LDZ;                     // [64][TR_LDZ] output gradient
    bf16* const Hs = D4 + TR_ROWS * TR_LDZ;                     // 3 x [64][TR_LD] activations -> gradients
    bf16* const Ws = Hs + 3 * TR_ROWS * TR_LD;                // the weights in use
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3, r0 = warp * 16;
    float* const prow = a.part + (long long)blockIdx.x * NPARAM;
    __shared__ double loss_w[4];
    __shared__ float bias_s[3 * HID + 2];  // b1..b3 and the output layer's two
    for (int e = tid; e < 3 * HID + 2; e += 128)
        bias_s[e] = e < 3 * HID ? a.bias[e / HID][e % HID] : a.bias[3][e - 3 * HID];
    double loss_acc = 0.0;
    const int n_slabs = (a.B + TR_ROWS - 1) / TR_ROWS;
    for (int slab = blockIdx.x; slab < n_slabs; slab += gridDim.x) {
        const bool first = slab == (int)blockIdx.x;
        const int b0 = slab * TR_ROWS;
        // weights in use order W1, W2, W3, W4, Wt4, Wt3, Wt2, one at a time (the
        // other CTA on the SM computes meanwhile)
        __syncthreads();  // the previous slab is done with the buffers
        stage_matrix(Ws, a.W[0], HID, KIN, tid);
        cp_async_commit();
        for (int e = tid; e < TR_ROWS * KIN; e += 128) {
            const int r = e / KIN, c = e % KIN, b = b0 + r;
            float v = 0.f;
            if (b < a.B && c < NIN) v = (a.x[b * NIN + c] - a.center[c]) / a.half[c];
            Zs[r * TR_LDZ + c] = __float2bfloat16_rn(v);
        }
        // ---- forward.  One copy of each layer's code: a CTA runs the kernel's body
        // once per slab, so its instruction fetches grow with the code's length
#pragma unroll 1
        for (int l = 0; l < 4; ++l) {
            cp_async_wait<0>();
            __syncthreads();  // layer l's weights and inputs visible
            const bf16* in = l == 0 ? Zs : Hs + (l - 1) * TR_ROWS * TR_LD;
            const int ld_in = l == 0 ? TR_LDZ : TR_LD, K = l == 0 ? KIN : HID;
            if (l < 3) {
                float acc[HID / 8][4];
                rows_times_weights<HID / 8>(acc, in, ld_in, K, Ws, r0, lane);
                bf16* out = Hs + l * TR_ROWS * TR_LD;
#pragma unroll
                for (int ni = 0; ni < HID / 8; ++ni)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int row = r0 + g + (r >= 2 ? 8 : 0), col = ni * 8 + 2 * t4 + (r & 1);
                        const float v = b0 + row < a.B ? act_tanh(acc[ni][r] + bias_s[l * HID + col]) : 0.f;
                        out[row * TR_LD + col] = __float2bfloat16_rn(v);
                    }
            } else {
                float acc[NOUTP / 8][4];
                rows_times_weights<NOUTP / 8>(acc, in, ld_in, K, Ws, r0, lane);
                // the loss and its gradient: columns 0 (stress / scale) and 1 (logit) of
                // n-tile 0 sit with the t4 == 0 lanes
                for (int e = lane; e < 16 * TR_LDZ; e += 32)
                    D4[(r0 + e / TR_LDZ) * TR_LDZ + e % TR_LDZ] = __float2bfloat16_rn(0.f);
                __syncwarp();
                if (t4 == 0) {
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int row = r0 + g + 8 * h2, b = b0 + row;
                        if (b >= a.B) continue;
                        const float y0 = acc[0][2 * h2] + bias_s[3 * HID], y1 = acc[0][2 * h2 + 1] + bias_s[3 * HID + 1];
                        const float t = a.target[b] * a.inv_scale, lab = a.label[b];
                        const float e = y0 - t;
                        loss_acc += (double)(e * e) + (double)a.lam * (double)bce_logits(y1, lab);
                        const float sg = 1.f / (1.f + expf(-y1));
                        D4[row * TR_LDZ + 0] = __float2bfloat16_rn(2.f * e / (float)a.B);
                        D4[row * TR_LDZ + 1] = __float2bfloat16_rn(a.lam * (sg - lab) / (float)a.B);
                    }
                }
            }
            __syncthreads();  // every warp is done with the weights (and, after layer 4, D4 and H3 are complete)
            if (l < 3)
                stage_matrix(Ws, a.W[l + 1], layer_def(l + 1).out_p, layer_def(l + 1).in_p, tid);
            else
                stage_matrix(Ws, a.Wt[3], HID, NOUTP, tid);  // Wt4 [128][16]
            cp_async_commit();
        }
        // ---- backward, layer 4: dW4 (16 x 128) from D4 and H3, db4
        bf16* const H1 = Hs;
        bf16* const H3 = Hs + 2 * TR_ROWS * TR_LD;
        {
            float acc[1][4][4];
            slab_outer<1, 4>(acc, D4, TR_LDZ, 0, H3, TR_LD, warp * 32, lane);
            put_wgrad<1, 4, 3>(prow, acc, OFF_W4, 0, warp * 32, g, t4, first);
            put_bgrad(prow, D4, TR_LDZ, 3, tid, first);
        }
        cp_async_wait<0>();  // Wt4
        __syncthreads();     // H3 read by every warp's dW4; Wt4 visible
        back_rows<HID / 8>(D4, TR_LDZ, NOUTP, Ws, H3, r0, g, t4, b0, a.B);  // D3 over H3
        __syncthreads();  // D3 complete; the weight buffer is free
        // layers 3 and 2 (index l = 2, 1) share one copy of the code: dW_l from D_l
        // (over H_l) and H_{l-1}, then D_{l-1} over H_{l-1} with Wt_l
        static_assert(layer_def(1).in == layer_def(2).in && layer_def(1).out == layer_def(2).out,
                      "the two hidden-to-hidden layers have one shape");
#pragma unroll 1
        for (int l = 2; l >= 1; --l) {
            bf16* const Dl = Hs + l * TR_ROWS * TR_LD;
            bf16* const Hp = Hs + (l - 1) * TR_ROWS * TR_LD;
            stage_matrix(Ws, a.Wt[l], HID, HID, tid);
            cp_async_commit();
            {
                float acc[2][HID / 8][4];
                slab_outer<2, HID / 8>(acc, Dl, TR_LD, warp * 32, Hp, TR_LD, 0, lane);
                put_wgrad<2, HID / 8, 1>(prow, acc, layer_def(l).offW, warp * 32, 0, g, t4, first);
                put_bgrad(prow, Dl, TR_LD, l, tid, first);
            }
            cp_async_wait<0>();  // Wt_l
            __syncthreads();
            back_rows<HID / 8>(Dl, TR_LD, HID, Ws, Hp, r0, g, t4, b0, a.B);
            __syncthreads();
        }
        // layer 1: dW1 (128 x 16) from D1 and the inputs
        {
            float acc[2][KIN / 8][4];
            slab_outer<2, KIN / 8>(acc, H1, TR_LD, warp * 32, Zs, TR_LDZ, 0, lane);
            put_wgrad<2, KIN / 8, 0>(prow, acc, OFF_W1, warp * 32, 0, g, t4, first);
            put_bgrad(prow, H1, TR_LD, 0, tid, first);
        }
    }
    // the CTA's loss: lane sums, then warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_down_sync(0xffffffffu, loss_acc, o);
    if (lane == 0) loss_w[warp] = loss_acc;
    __syncthreads();
    if (tid == 0) a.loss_part[blockIdx.x] = (loss_w[0] + loss_w[1]) + (loss_w[2] + loss_w[3]);
}

// Sums the CTAs' partial rows in order.  mode 0: gradient into grad.  mode 1: an
// Adam step on the FP32 masters p (m, v its moments) and the refreshed BF16
// weight copies and FP32 biases of that parameter.  Thread 0 of block 0 also
// finishes the loss (mean over the batch).
struct FinishArgs {
    const float* part;
    const double* loss_part;
    int n_rows, B;
    float* grad;
    float *p, *m, *v;
    float lr, b1, b2, eps, c1, c2;
    bf16* W[4];
    bf16* Wt[4];
    float* bias[4];
    float* loss_f;
    double* loss_d;
};

constexpr int FIN_PARAMS = 64, FIN_SPLIT = 4;  // parameters per block, threads per parameter
__global__ void __launch_bounds__(FIN_PARAMS * FIN_SPLIT) grad_finish_kernel(FinishArgs a, int mode)
{
    // thread (q, j): parameter k = blockIdx.x * FIN_PARAMS + j, rows c = q, q + 4, ...
    // in eight interleaved sums; the four quarters combine in a fixed order
    const int j = threadIdx.x % FIN_PARAMS, q = threadIdx.x / FIN_PARAMS;
    const long long k = (long long)blockIdx.x * FIN_PARAMS + j;
    __shared__ float quarter[FIN_SPLIT][FIN_PARAMS];
    if (k < NPARAM) {
        float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int c = q;
        for (; c + 7 * FIN_SPLIT < a.n_rows; c += 8 * FIN_SPLIT)
#pragma unroll
            for (int u = 0; u < 8; ++u) s8[u] += a.part[(long long)(c + u * FIN_SPLIT) * NPARAM + k];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c + u * FIN_SPLIT < a.n_rows) s8[u] += a.part[(long long)(c + u * FIN_SPLIT) * NPARAM + k];
        quarter[q][j] = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
    }
    __syncthreads();
    if (blockIdx.x == 0 && q == 1 && j < 32) {
        // the loss, by one otherwise idle warp: lane sums over rows lane, lane + 32, ...,
        // then a butterfly over the lanes (a fixed order, so the same every call)
        double s = 0.0;
        for (int c = j; c < a.n_rows; c += 32) s += a.loss_part[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (j == 0) {
            s /= (double)a.B;
            if (a.loss_f) *a.loss_f = (float)s;
            if (a.loss_d) *a.loss_d = s;
        }
        return;
    }
    if (q != 0 || k >= NPARAM) return;
    const float gk = (quarter[0][j] + quarter[1][j]) + (quarter[2][j] + quarter[3][j]);
    if (mode == 0) {
        a.grad[k] = gk;
        return;
    }
    const float mk = a.b1 * a.m[k] + (1.f - a.b1) * gk;
    const float vk = a.b2 * a.v[k] + (1.f - a.b2) * gk * gk;
    a.m[k] = mk;
    a.v[k] = vk;
    const float pk = a.p[k] - a.lr * (mk * a.c1) / (sqrtf(vk * a.c2) + a.eps);
    a.p[k] = pk;
    for (int l = 0; l < 4; ++l) {  // the parameter's BF16 weight entries or FP32 bias
        const LayerDef L = layer_def(l);
        if (k >= L.offW && k < L.offB) {
            const int o = (int)((k - L.offW) / L.in), i = (int)((k - L.offW) % L.in);
            const bf16 hv = __float2bfloat16_rn(pk);
            a.W[l][o * L.in_p + i] = hv;
            a.Wt[l][i * L.out_p + o] = hv;
        } else if (k >= L.offB && k < L.offB + L.out) {
            a.bias[l][k - L.offB] = pk;
        }
    }
}

struct mlp_handle {
    mlp_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int bbuf = 0;  // batch rows of the buffers (max_batch rounded up to 64)
    int splits = 0;
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr;
    bf16 *W[4] = {}, *Wt[4] = {};
    float* bias[4] = {};
    bf16 *Z = nullptr, *Zt = nullptr;
    bf16 *H[3] = {}, *Ht[3] = {};
    float* OUT = nullptr;
    float* part = nullptr;         // [tr_rows][NPARAM] partial gradients of train_fused_kernel
    int tr_rows = 0;               // its CTAs at most (one partial row each)
    double* loss_part = nullptr;   // [tr_rows]
    double* loss_d = nullptr;
    float *center = nullptr, *half = nullptr;
    int* over_budget = nullptr;  // [MAX_BINS]
    int n_bins = 0;
    float ls_lo = 0.f, ls_hi = 1.f;
    long long adam_t = 0;
    long long launches = 0;
    std::vector<void*> allocs;
};

namespace {

void release(mlp_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

template <class T>
cudaError_t alloc(mlp_handle* h, T** p, size_t n)
{
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) {
        h->allocs.push_back(*p);
        e = cudaMemsetAsync(*p, 0, n * sizeof(T), h->stream);
    }
    return e;
}

int rows8(int B) { return (B + 7) / 8 * 8; }

template <int EPI>
cudaError_t gemm(mlp_handle* h, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int kchunk,
                 const Epi& ep)
{
    const int splits = (K + kchunk - 1) / kchunk;
    dim3 grid((M + 63) / 64, (N + 63) / 64, splits);
    gemm_nt<EPI><<<grid, 128, 0, h->stream>>>(A, lda, B, ldb, M, N, K, kchunk, ep);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t forward(mlp_handle* h, const float* x, int B)
{
    const int Br = rows8(B), bb = h->bbuf;
    normalise_kernel<<<(bb + 127) / 128, 128, 0, h->stream>>>(x, B, bb, h->center, h->half, h->Z, h->Zt);
    h->launches++;
    const bf16* in = h->Z;
    int ld_in = KIN;
    for (int l = 0; l < 4; ++l) {
        const LayerDef L = layer_def(l);
        Epi ep{};
        ep.bias = h->bias[l];
        ep.rows_live = B;
        ep.rows_buf = bb;
        cudaError_t e;
        if (l < 3) {
            ep.out_b = h->H[l];
            ep.out_t = h->Ht[l];
            ep.ld_out = HID;
            ep.ld_t = bb;
            e = gemm<EPI_TANH>(h, in, ld_in, h->W[l], L.in_p, Br, L.out_p, L.in_p, L.in_p, ep);
            in = h->H[l];
            ld_in = HID;
        } else {
            ep.out_f = h->OUT;
            ep.ld_out = NOUTP;
            e = gemm<EPI_OUT>(h, in, ld_in, h->W[l], L.in_p, Br, L.out_p, L.in_p, L.in_p, ep);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Loss, gradient (mode 0: into h->G) or gradient and Adam step (mode 1): the
// fused training kernel over slabs of 64 rows, then the ordered reduction.
cudaError_t fused_step(mlp_handle* h, const float* x, const float* target, const float* label, int B, int mode,
                       float* loss_f, double* loss_d)
{
    TrainArgs ta{};
    ta.x = x;
    ta.target = target;
    ta.label = label;
    ta.B = B;
    for (int l = 0; l < 4; ++l) {
        ta.W[l] = h->W[l];
        ta.Wt[l] = h->Wt[l];
        ta.bias[l] = h->bias[l];
    }
    ta.center = h->center;
    ta.half = h->half;
    ta.inv_scale = (float)(1.0 / h->cfg.sigma_scale);
    ta.lam = (float)h->cfg.lam;
    ta.part = h->part;
    ta.loss_part = h->loss_part;
    const int slabs = (B + TR_ROWS - 1) / TR_ROWS;
    const int rows = slabs < h->tr_rows ? slabs : h->tr_rows;  // every CTA gets at least one slab
    train_fused_kernel<<<rows, 128, TR_SMEM, h->stream>>>(ta);
    h->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    FinishArgs fa{};
    fa.part = h->part;
    fa.loss_part = h->loss_part;
    fa.n_rows = rows;
    fa.B = B;
    fa.grad = h->G;
    fa.p = h->P;
    fa.m = h->M;
    fa.v = h->V;
    if (mode == 1) {
        h->adam_t++;
        const double b1 = h->cfg.beta1, b2 = h->cfg.beta2;
        fa.lr = (float)h->cfg.lr;
        fa.b1 = (float)b1;
        fa.b2 = (float)b2;
        fa.eps = (float)h->cfg.eps;
        fa.c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)h->adam_t)));
        fa.c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)h->adam_t)));
    }
    for (int l = 0; l < 4; ++l) {
        fa.W[l] = h->W[l];
        fa.Wt[l] = h->Wt[l];
        fa.bias[l] = h->bias[l];
    }
    fa.loss_f = loss_f;
    fa.loss_d = loss_d;
    grad_finish_kernel<<<(int)((NPARAM + FIN_PARAMS - 1) / FIN_PARAMS), FIN_PARAMS * FIN_SPLIT, 0, h->stream>>>(fa,
                                                                                                         mode);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t refresh(mlp_handle* h)
{
    int total = 0;
    for (int l = 0; l < 4; ++l) total += layer_def(l).out_p * layer_def(l).in_p + layer_def(l).out_p;
    refresh_kernel<<<(total + 255) / 256, 256, 0, h->stream>>>(h->P, h->W[0], h->Wt[0], h->W[1], h->Wt[1], h->W[2],
                                                                h->Wt[2], h->W[3], h->Wt[3], h->bias[0], h->bias[1],
                                                                h->bias[2], h->bias[3]);
    h->launches++;
    return cudaGetLastError();
}

lb_status invalid(const char* msg)
{
    lbhb::set_handleless_error(msg);
    return LB_ERR_INVALID;
}

lb_status check_batch(const mlp_handle* h, int B)
{
    if (B >= 1 && B <= h->cfg.max_batch) return LB_OK;
    char buf[128];
    snprintf(buf, sizeof buf, "mlp: batch %d outside 1..max_batch (%d)", B, h->cfg.max_batch);
    lbhb::set_handleless_error(buf);
    return LB_ERR_INVALID;
}

}  // namespace

extern "C" {

long long mlp_param_count(void) { return NPARAM; }

lb_status mlp_create(const mlp_config* cfg, void* cuda_stream, mlp_handle** out)
{
    if (!out || !cfg) return invalid("mlp_create: NULL config or output");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > (1 << 24) || !(cfg->sigma_scale > 0.0) || !(cfg->lr >= 0.0))
        return invalid("mlp_create: max_batch, sigma_scale or lr out of range");
    for (int c = 0; c < NIN; ++c)
        if (!(cfg->half_range[c] > 0.0) || !std::isfinite(cfg->center[c]))
            return invalid("mlp_create: half_range must be > 0 and center finite");
    mlp_handle* h = new (std::nothrow) mlp_handle();
    if (!h) return LB_ERR_NOMEM;
    h->cfg = *cfg;
    cudaGetDevice(&h->device);
    cudaError_t e = cudaSuccess;
    if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = e == cudaSuccess;
    }
    h->bbuf = (cfg->max_batch + 63) / 64 * 64;
    const int bb = h->bbuf;
    h->tr_rows = std::min(TR_MAX_CTAS, bb / TR_ROWS);
    if (e == cudaSuccess) e = alloc(h, &h->P, NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->M, NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->V, NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->G, NPARAM);
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        e = alloc(h, &h->W[l], (size_t)layer_def(l).out_p * layer_def(l).in_p);
        if (e == cudaSuccess) e = alloc(h, &h->Wt[l], (size_t)layer_def(l).out_p * layer_def(l).in_p);
        if (e == cudaSuccess) e = alloc(h, &h->bias[l], (size_t)layer_def(l).out_p);
    }
    if (e == cudaSuccess) e = alloc(h, &h->Z, (size_t)bb * KIN);
    if (e == cudaSuccess) e = alloc(h, &h->Zt, (size_t)bb * KIN);
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        e = alloc(h, &h->H[l], (size_t)bb * HID);
        if (e == cudaSuccess) e = alloc(h, &h->Ht[l], (size_t)bb * HID);
    }
    if (e == cudaSuccess) e = alloc(h, &h->OUT, (size_t)bb * NOUTP);
    if (e == cudaSuccess) e = alloc(h, &h->part, (size_t)h->tr_rows * NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->loss_part, (size_t)h->tr_rows);
    if (e == cudaSuccess) e = alloc(h, &h->loss_d, 1);
    if (e == cudaSuccess) e = alloc(h, &h->center, NIN);
    if (e == cudaSuccess) e = alloc(h, &h->half, NIN);
    if (e == cudaSuccess)  // the fused serving kernel keeps activations and weights in shared memory
        e = cudaFuncSetAttribute(serve_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SRV_SMEM);
    if (e == cudaSuccess)  // and so does the fused training kernel
        e = cudaFuncSetAttribute(train_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM);
    if (e == cudaSuccess) e = alloc(h, &h->over_budget, MAX_BINS);
    if (e == cudaSuccess) {
        float c[NIN], hr[NIN];
        for (int i = 0; i < NIN; ++i) {
            c[i] = (float)cfg->center[i];
            hr[i] = (float)cfg->half_range[i];
        }
        e = cudaMemcpyAsync(h->center, c, sizeof c, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->half, hr, sizeof hr, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(h);
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    *out = h;
    return LB_OK;
}

lb_status mlp_set_params(mlp_handle* h, const float* params, long long n)
{
    if (!h || !params || n != NPARAM) return invalid("mlp: NULL handle or parameters, or wrong count");
    cudaError_t e = cudaMemcpyAsync(h->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->M, 0, sizeof(float) * NPARAM, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->V, 0, sizeof(float) * NPARAM, h->stream);
    if (e == cudaSuccess) e = refresh(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->adam_t = 0;
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_get_params(mlp_handle* h, float* params, long long n)
{
    if (!h || !params || n != NPARAM) return invalid("mlp: NULL handle or parameters, or wrong count");
    cudaError_t e = cudaMemcpyAsync(params, h->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_forward(mlp_handle* h, const float* x, int batch, float* out)
{
    if (!h || !x || !out) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    cudaError_t e = forward(h, x, batch);
    if (e == cudaSuccess) {
        output_kernel<<<(batch + 255) / 256, 256, 0, h->stream>>>(h->OUT, batch, (float)h->cfg.sigma_scale, out);
        h->launches++;
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_gradients(mlp_handle* h, const float* x, const float* target_stress, const float* label, int batch,
                        float* grad, double* loss)
{
    if (!h || !x || !target_stress || !label || !grad) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    cudaError_t e = fused_step(h, x, target_stress, label, batch, 0, nullptr, h->loss_d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, h->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream);
    double l = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, h->loss_d, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (loss) *loss = l;
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_train_step(mlp_handle* h, const float* x, const float* target_stress, const float* label, int batch,
                         float* loss_dev)
{
    if (!h || !x || !target_stress || !label) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    const cudaError_t e = fused_step(h, x, target_stress, label, batch, 1, loss_dev, nullptr);
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_serve(mlp_handle* h, const float* x, int batch, float* stress, float* logit, int* fallback)
{
    if (!h || !x || !stress || !logit || !fallback) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    ServeArgs a{};
    a.x = x;
    a.B = batch;
    for (int l = 0; l < 4; ++l) {
        a.W[l] = h->W[l];
        a.bias[l] = h->bias[l];
    }
    a.center = h->center;
    a.half = h->half;
    a.scale = (float)h->cfg.sigma_scale;
    a.margin = (float)h->cfg.logit_margin;
    a.over_budget = h->over_budget;
    a.n_bins = h->n_bins;
    a.ls_lo = h->ls_lo;
    a.ls_hi = h->ls_hi;
    a.stress = stress;
    a.logit = logit;
    a.fallback = fallback;
    serve_fused_kernel<<<(batch + SRV_ROWS - 1) / SRV_ROWS, 128, SRV_SMEM, h->stream>>>(a);
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_set_error_budget(mlp_handle* h, const float* bin_error, int n_bins, double log_s_lo,
                               double log_s_hi, double budget)
{
    if (!h || n_bins < 0 || n_bins > MAX_BINS || (n_bins > 0 && (!bin_error || !(log_s_hi > log_s_lo))))
        return invalid("mlp_set_error_budget: NULL handle, n_bins outside 0..256 or empty log S range");
    int flags[MAX_BINS] = {0};
    for (int k = 0; k < n_bins; ++k) flags[k] = !(bin_error[k] <= budget);  // NaN error is over budget
    cudaError_t e = cudaMemcpyAsync(h->over_budget, flags, sizeof(int) * MAX_BINS, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LB_ERR_CUDA;
    h->n_bins = n_bins;
    h->ls_lo = (float)log_s_lo;
    h->ls_hi = (float)log_s_hi;
    return LB_OK;
}

long long mlp_kernel_launches(const mlp_handle* h) { return h ? h->launches : 0; }

void mlp_destroy(mlp_handle* h) { release(h); }

}  // extern "C"
